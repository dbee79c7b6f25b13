// SPH pair sums over cell lists: summation density (rho^n of Eq. 19, with
// the equation of state) and the gas pressure (+ artificial viscosity)
// acceleration of the first term of Eq. 19, with the adiabatic energy rate.
//
// One thread per particle in cell order. Candidates are read from the
// contiguous particle ranges of rows of cells (keys are x-fastest, so the
// cells of one row within the reach form one range). Rows and row ends whose
// slab lies farther than 2h (plus a rounding margin) from the particle are
// skipped. Neighbour membership r^2 < 4h^2 is evaluated with explicitly
// rounded operations so that it is a plain IEEE decision.
#include "tfsph_internal.cuh"

namespace tfsph {
namespace {

// Distance, in cell units, from a particle at fractional cell position f to
// the slab of the cell o cells away along one axis (0 for its own cell).
template <class T> __device__ __forceinline__ T slab_dist(int o, T f)
{
    if (o > 0) return fmax(T(0), T(o) - f);
    if (o < 0) return fmax(T(0), f + T(-o) - T(1));
    return T(0);
}

// Wraps (periodic) or rejects (open) a cell coordinate; -1 when outside.
__device__ __forceinline__ int axis_wrap(int c, int n, int per)
{
    if (c >= 0 && c < n) return c;
    if (!per) return -1;
    return c < 0 ? c + n : c - n;
}

// Candidate neighbours of one row of cells: up to three contiguous storage
// ranges (the main window and, on a periodic axis, the parts wrapped around
// either end), visited as one index space so that the pair loop has a single
// call site.
struct RowRanges {
    uint32_t b0, n0;  // wrapped part below 0
    uint32_t b1, n1;  // wrapped part above n-1
    uint32_t b2, n2;  // main window
    __device__ __forceinline__ uint32_t total() const { return n0 + n1 + n2; }
    __device__ __forceinline__ uint32_t at(uint32_t i) const
    {
        return i < n0 ? b0 + i : (i < n0 + n1 ? b1 + (i - n0) : b2 + (i - n0 - n1));
    }
};

// Calls f(RowRanges) once for every row of cells (fixed y, z) that may hold
// neighbours of a particle at (px, py, pz).
template <class T, int DIM, class F>
__device__ __forceinline__ void for_each_row(const Geo<T> &G, const uint32_t *__restrict__ start,
                                             T px, T py, T pz, F &&f)
{
    T tx, ty = T(0), tz = T(0);
    const int cx = axis_cell(px, G.lo[0], G.inv_w[0], G.n[0], tx);
    const int cy = DIM > 1 ? axis_cell(py, G.lo[1], G.inv_w[1], G.n[1], ty) : 0;
    const int cz = DIM > 2 ? axis_cell(pz, G.lo[2], G.inv_w[2], G.n[2], tz) : 0;
    const T fx = tx - T(cx);
    const T fy = DIM > 1 ? ty - T(cy) : T(0);
    const T fz = DIM > 2 ? tz - T(cz) : T(0);

    const int zlo = DIM > 2 ? (G.full[2] ? 0 : -G.R[2]) : 0;
    const int zhi = DIM > 2 ? (G.full[2] ? G.n[2] - 1 : G.R[2]) : 0;
    const int ylo = DIM > 1 ? (G.full[1] ? 0 : -G.R[1]) : 0;
    const int yhi = DIM > 1 ? (G.full[1] ? G.n[1] - 1 : G.R[1]) : 0;
    const int nx = G.n[0];

#pragma unroll 1
    for (int oz = zlo; oz <= zhi; ++oz) {
        int z = 0;
        T dz2 = T(0);
        if (DIM > 2) {
            if (G.full[2]) {
                z = oz;
            } else {
                z = axis_wrap(cz + oz, G.n[2], G.per[2]);
                if (z < 0) continue;
                const T s = slab_dist(oz, fz) * G.w[2];
                dz2 = s * s;
                if (dz2 >= G.lim2) continue;
            }
        }
#pragma unroll 1
        for (int oy = ylo; oy <= yhi; ++oy) {
            int y = 0;
            T dy2 = T(0);
            if (DIM > 1) {
                if (G.full[1]) {
                    y = oy;
                } else {
                    y = axis_wrap(cy + oy, G.n[1], G.per[1]);
                    if (y < 0) continue;
                    const T s = slab_dist(oy, fy) * G.w[1];
                    dy2 = s * s;
                    if (dz2 + dy2 >= G.lim2) continue;
                }
            }
            const uint32_t row = (uint32_t)nx * ((uint32_t)y + (uint32_t)G.n[1] * (uint32_t)z);
            RowRanges rr;
            rr.n0 = rr.n1 = 0;
            rr.b0 = rr.b1 = 0;
            if (G.full[0]) {
                rr.b2 = start[row];
                rr.n2 = start[row + nx] - rr.b2;
            } else {
                const T rem = G.lim2 - dz2 - dy2;
                int ohi = 0, olo = 0;
#pragma unroll 1
                for (int o = 1; o <= G.R[0]; ++o) {
                    const T s = slab_dist(o, fx) * G.w[0];
                    if (s * s < rem) ohi = o; else break;
                }
#pragma unroll 1
                for (int o = 1; o <= G.R[0]; ++o) {
                    const T s = slab_dist(-o, fx) * G.w[0];
                    if (s * s < rem) olo = -o; else break;
                }
                int x0 = cx + olo, x1 = cx + ohi;
                if (G.per[0]) {
                    if (x0 < 0) {
                        rr.b0 = start[row + x0 + nx];
                        rr.n0 = start[row + nx] - rr.b0;
                        x0 = 0;
                    }
                    if (x1 >= nx) {
                        rr.b1 = start[row];
                        rr.n1 = start[row + (x1 - nx) + 1] - rr.b1;
                        x1 = nx - 1;
                    }
                } else {
                    if (x0 < 0) x0 = 0;
                    if (x1 >= nx) x1 = nx - 1;
                }
                rr.b2 = start[row + x0];
                rr.n2 = start[row + x1 + 1] - rr.b2;
            }
            f(rr);
        }
    }
}

// Squared pair distance with minimum image; d[] receives x_a - x_b.
template <class T, int DIM>
__device__ __forceinline__ T pair_r2(const Geo<T> &G, const V4<T> &pa, const V4<T> &pb, T d[3])
{
    d[0] = min_image(sub_rn(pa.x, pb.x), G.per[0], G.L[0], G.halfL[0]);
    T r2 = mul_rn(d[0], d[0]);
    if (DIM > 1) {
        d[1] = min_image(sub_rn(pa.y, pb.y), G.per[1], G.L[1], G.halfL[1]);
        r2 = add_rn(r2, mul_rn(d[1], d[1]));
    } else {
        d[1] = T(0);
    }
    if (DIM > 2) {
        d[2] = min_image(sub_rn(pa.z, pb.z), G.per[2], G.L[2], G.halfL[2]);
        r2 = add_rn(r2, mul_rn(d[2], d[2]));
    } else {
        d[2] = T(0);
    }
    return r2;
}

// rho_a = m sum_b W(r_ab, h), self term included. For gas, also p_a/rho_a^2
// into pos[a].w (isothermal p = cs^2 rho, adiabatic p = (gamma-1) rho e).
template <class T, int DIM, bool STATS>
__global__ void __launch_bounds__(128, 1)
k_density(Geo<T> G, Phys<T> Ph, const V4<T> *__restrict__ pos, const V4<T> *__restrict__ vel,
          const uint32_t *__restrict__ id, const uint32_t *__restrict__ start, int n, T mass,
          T *__restrict__ rho_out, T *pr_out, int32_t *__restrict__ cnt, uint64_t *__restrict__ fpr)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const V4<T> pa = pos[a];
    T sum = T(0);
    int c = 0;
    uint64_t fp = 0;
    for_each_row<T, DIM>(G, start, pa.x, pa.y, pa.z, [&](const RowRanges &rr) {
        const uint32_t tot = rr.total();
        for (uint32_t i = 0; i < tot; ++i) {
            const uint32_t b = rr.at(i);
            const V4<T> pb = pos[b];
            T d[3];
            const T r2 = pair_r2<T, DIM>(G, pa, pb, d);
            if (r2 < G.h2x4) {
                sum += kernel_w(G, sqrt(r2) * G.inv_h);
                if (STATS) {
                    ++c;
                    fp += (uint64_t)((id[b] & kIdMask) + 1u) * 0x9E3779B97F4A7C15ull;
                }
            }
        }
    });
    const T r = mass * sum;
    rho_out[a] = r;
    if (pr_out) {
        const T pr = Ph.eos == TFSPH_EOS_ADIABATIC ? Ph.gm1 * vel[a].w / r : Ph.cs2 / r;
        pr_out[4 * (size_t)a + 3] = pr;  // .w of pos[a]; the other lanes are untouched
    }
    if (STATS) {
        cnt[a] = c;
        fpr[a] = fp;
    }
}

// A_a = -m sum_b (p_a/rho_a^2 + p_b/rho_b^2 + Pi_ab) grad_a W_ab and
// de_a/dt = m sum_b (p_a/rho_a^2 + Pi_ab/2) v_ab . grad_a W_ab, with
// grad_a W_ab = (r_a - r_b) (1/r) dW/dr and Monaghan's
// Pi_ab = (-alpha cbar mu + beta mu^2) / rhobar for v_ab . r_ab < 0,
// mu = h v_ab . r_ab / (r^2 + 0.01 h^2). FULL = false: isothermal gas
// without viscosity (positions and p/rho^2 only).
template <class T, int DIM, bool FULL>
__global__ void __launch_bounds__(128, 1)
k_force(Geo<T> G, Phys<T> Ph, const V4<T> *__restrict__ pos, const V4<T> *__restrict__ vel,
        const T *__restrict__ rho, const uint32_t *__restrict__ start, int n, V4<T> *__restrict__ acc)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const V4<T> pa = pos[a];
    V4<T> va;
    T rhoa = T(1), ca = Ph.cs;
    if (FULL) {
        va = vel[a];
        rhoa = rho[a];
        if (Ph.eos == TFSPH_EOS_ADIABATIC) ca = sqrt(Ph.gamma * Ph.gm1 * va.w);
    }
    const T qa = pa.w;
    T ax = T(0), ay = T(0), az = T(0), de = T(0);
    for_each_row<T, DIM>(G, start, pa.x, pa.y, pa.z, [&](const RowRanges &rr) {
        const uint32_t tot = rr.total();
        for (uint32_t i = 0; i < tot; ++i) {
            const uint32_t b = rr.at(i);
            const V4<T> pb = pos[b];
            T d[3];
            const T r2 = pair_r2<T, DIM>(G, pa, pb, d);
            if (!(r2 < G.h2x4)) continue;
            const T F = kernel_f(G, sqrt(r2) * G.inv_h);  // (1/r) dW/dr
            T coef = qa + pb.w;
            if (FULL) {
                const V4<T> vb = vel[b];
                const T vx = va.x - vb.x;
                const T vy = DIM > 1 ? va.y - vb.y : T(0);
                const T vz = DIM > 2 ? va.z - vb.z : T(0);
                const T vr = vx * d[0] + vy * d[1] + vz * d[2];
                T pi = T(0);
                if (Ph.av && vr < T(0)) {
                    const T mu = Ph.h * vr / (r2 + Ph.eta2);
                    const T cb = Ph.eos == TFSPH_EOS_ADIABATIC ? sqrt(Ph.gamma * Ph.gm1 * vb.w) : Ph.cs;
                    const T cbar = T(0.5) * (ca + cb);
                    const T rbar = T(0.5) * (rhoa + rho[b]);
                    pi = (-Ph.av_alpha * cbar * mu + Ph.av_beta * mu * mu) / rbar;
                }
                coef += pi;
                de += (qa + T(0.5) * pi) * vr * F;
            }
            const T s = coef * F;
            ax -= s * d[0];
            if (DIM > 1) ay -= s * d[1];
            if (DIM > 2) az -= s * d[2];
        }
    });
    V4<T> out;
    out.x = Ph.m_g * ax;
    out.y = Ph.m_g * ay;
    out.z = Ph.m_g * az;
    out.w = Ph.m_g * de;
    acc[a] = out;
}

template <class T, int DIM>
cudaError_t density_t(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &P, void *rho,
                      bool gas, int32_t *cnt, uint64_t *fprint)
{
    if (P.n == 0) return cudaSuccess;
    const Geo<T> &G = *static_cast<const Geo<T> *>(geo);
    const Phys<T> &Ph = *static_cast<const Phys<T> *>(phys);
    const int n = (int)P.n;
    const int threads = 128;
    const int blocks = (n + threads - 1) / threads;
    auto *pos = static_cast<V4<T> *>(P.pos[P.cur]);
    auto *vel = static_cast<const V4<T> *>(P.vel[P.cur]);
    T *pr = gas ? reinterpret_cast<T *>(pos) : nullptr;
    const T mass = gas ? Ph.m_g : Ph.m_d;
    if (cnt) {
        k_density<T, DIM, true><<<blocks, threads, 0, L.stream>>>(G, Ph, pos, vel, P.id[P.cur], P.start, n,
                                                                  mass, static_cast<T *>(rho), pr, cnt, fprint);
    } else {
        k_density<T, DIM, false><<<blocks, threads, 0, L.stream>>>(G, Ph, pos, vel, P.id[P.cur], P.start, n,
                                                                   mass, static_cast<T *>(rho), pr, nullptr, nullptr);
    }
    return cudaGetLastError();
}

template <class T, int DIM>
cudaError_t force_t(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &P, const void *rho,
                    void *acc)
{
    if (P.n == 0) return cudaSuccess;
    const Geo<T> &G = *static_cast<const Geo<T> *>(geo);
    const Phys<T> &Ph = *static_cast<const Phys<T> *>(phys);
    const int n = (int)P.n;
    const int threads = 128;
    const int blocks = (n + threads - 1) / threads;
    auto *pos = static_cast<const V4<T> *>(P.pos[P.cur]);
    auto *vel = static_cast<const V4<T> *>(P.vel[P.cur]);
    const bool full = Ph.av || Ph.eos == TFSPH_EOS_ADIABATIC;
    if (full) {
        k_force<T, DIM, true><<<blocks, threads, 0, L.stream>>>(G, Ph, pos, vel, static_cast<const T *>(rho),
                                                                P.start, n, static_cast<V4<T> *>(acc));
    } else {
        k_force<T, DIM, false><<<blocks, threads, 0, L.stream>>>(G, Ph, pos, vel, static_cast<const T *>(rho),
                                                                 P.start, n, static_cast<V4<T> *>(acc));
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_density(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &P, void *rho,
                           bool gas, int32_t *cnt, uint64_t *fprint)
{
    if (L.precision == TFSPH_FP64) {
        switch (L.dim) {
            case 1: return density_t<double, 1>(L, geo, phys, P, rho, gas, cnt, fprint);
            case 2: return density_t<double, 2>(L, geo, phys, P, rho, gas, cnt, fprint);
            default: return density_t<double, 3>(L, geo, phys, P, rho, gas, cnt, fprint);
        }
    }
    switch (L.dim) {
        case 1: return density_t<float, 1>(L, geo, phys, P, rho, gas, cnt, fprint);
        case 2: return density_t<float, 2>(L, geo, phys, P, rho, gas, cnt, fprint);
        default: return density_t<float, 3>(L, geo, phys, P, rho, gas, cnt, fprint);
    }
}

cudaError_t launch_force(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G, const void *rho,
                         void *acc)
{
    if (L.precision == TFSPH_FP64) {
        switch (L.dim) {
            case 1: return force_t<double, 1>(L, geo, phys, G, rho, acc);
            case 2: return force_t<double, 2>(L, geo, phys, G, rho, acc);
            default: return force_t<double, 3>(L, geo, phys, G, rho, acc);
        }
    }
    switch (L.dim) {
        case 1: return force_t<float, 1>(L, geo, phys, G, rho, acc);
        case 2: return force_t<float, 2>(L, geo, phys, G, rho, acc);
        default: return force_t<float, 3>(L, geo, phys, G, rho, acc);
    }
}

}  // namespace tfsph
