// SPH pair sums over cell lists: summation density (rho^n of Eq. 19, with
// the equation of state) and the gas pressure (+ artificial viscosity)
// acceleration of the first term of Eq. 19, with the adiabatic energy rate.
//
// Tiled path (default). One CTA owns a box of cells. It stages the particles
// of the box and of its halo (the cells within the search reach R) into
// shared memory once, with a local table of cell starts, and then each thread
// takes one owned particle and walks its candidate rows in shared memory.
// Rows and row ends whose slab lies farther than 2h (plus a rounding margin)
// from the particle are skipped. The halo cells that lie across a periodic
// seam are known per row segment, so the inner loop of the common case is a
// plain difference of coordinates; seam segments use the two-sum displacement
// below. A tile whose halo does not fit in shared memory computes from global
// memory with the same arithmetic.
//
// Neighbour membership r^2 < 4h^2 is evaluated with explicitly rounded
// operations so that it is a plain IEEE decision, the same one the checker
// takes.
#include <algorithm>
#include <cmath>

#include "tfsph_internal.cuh"

namespace tfsph {
namespace {

constexpr int kTileThreads = 256;

// ---------------------------------------------------------------------------
// Pair geometry
// ---------------------------------------------------------------------------

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

// Displacement x_a - x_b along one axis for the neighbour decision. Across
// the periodic seam (|s| > L/2) the image shift is applied to s, which is
// exact because s and L are within a factor of two, and the rounding error
// of s (Knuth's two-sum) is added back.
template <class T> __device__ __forceinline__ T disp(T xa, T xb, int per, T L, T half)
{
    const T s = sub_rn(xa, xb);
    if (per && (s > half || s < -half)) {
        const T bb = sub_rn(s, xa);
        const T e = add_rn(sub_rn(xa, sub_rn(s, bb)), sub_rn(-xb, bb));
        const T t = s > half ? sub_rn(s, L) : add_rn(s, L);
        return add_rn(t, e);
    }
    return s;
}

template <class T, int DIM, bool SEAM>
__device__ __forceinline__ T pair_r2(const Geo<T> &G, const V4<T> &pa, const V4<T> &pb, T d[3])
{
    d[0] = SEAM ? disp(pa.x, pb.x, G.per[0], G.L[0], G.halfL[0]) : sub_rn(pa.x, pb.x);
    T r2 = mul_rn(d[0], d[0]);
    if (DIM > 1) {
        d[1] = SEAM ? disp(pa.y, pb.y, G.per[1], G.L[1], G.halfL[1]) : sub_rn(pa.y, pb.y);
        r2 = fma_rn(d[1], d[1], r2);
    } else {
        d[1] = T(0);
    }
    if (DIM > 2) {
        d[2] = SEAM ? disp(pa.z, pb.z, G.per[2], G.L[2], G.halfL[2]) : sub_rn(pa.z, pb.z);
        r2 = fma_rn(d[2], d[2], r2);
    } else {
        d[2] = T(0);
    }
    return r2;
}

// Per-candidate data staged besides the position: a second V4 (velocity for
// the full force, lambda_A for the force adjoint) and/or one scalar (density
// for the full force, lambda_rho for the density adjoint).
template <int MODE> struct ModeUses {
    static constexpr bool vel = MODE == 3 || MODE == 4;
    static constexpr bool rho = MODE == 3 || MODE == 5;
};

// ---------------------------------------------------------------------------
// Per-pair work. MODE 0: density, 1: density + neighbour statistics,
// 2: isothermal force without viscosity, 3: force with viscosity and/or
// adiabatic energy rate, 4: adjoint of the isothermal force, 5: adjoint of
// the density.
//
// Adjoints (reverse mode, lambda_X = dLoss/dX), as gathers over neighbours:
//   A_a   = -m sum_b (q_a + q_b) F(r_ab) d_ab,  d_ab = x_a - x_b,
//           F = (1/r) dW/dr, q = p/rho^2;
//   lambda_q_a  = -m sum_b F_ab d_ab . (lambda_A_a - lambda_A_b)
//   lambda_x_a += -m sum_b (q_a + q_b) M(d_ab) (lambda_A_a - lambda_A_b),
//           M(d) v = F v + (F'(r)/r) (d . v) d
//   rho_a = m sum_b W(r_ab):
//   lambda_x_a += m sum_b F_ab d_ab (lambda_rho_a + lambda_rho_b)
// ---------------------------------------------------------------------------
template <class T, int MODE> struct PairAcc {
    // density
    T sum = T(0);
    int cnt = 0;
    uint64_t fp = 0;
    // force
    T qa = T(0), rhoa = T(1), ca = T(0);
    V4<T> va;
    T ax = T(0), ay = T(0), az = T(0), de = T(0);
    // adjoints: lambda_A_a (in va), lambda_rho_a (in rhoa); lambda_q in de,
    // lambda_x in ax, ay, az

    // candidate b: position (with p_b/rho_b^2 in .w), velocity, density, id,
    // squared distance r2 and displacement d = x_a - x_b
    __device__ __forceinline__ void add(const Geo<T> &G, const Phys<T> &Ph, const V4<T> &pb, const V4<T> *vb,
                                        T rhob, uint32_t idb, T r2, const T d[3])
    {
        if (!(r2 < G.h2x4)) return;
        if (MODE == 4 || MODE == 5) {
            if (r2 == T(0)) return;  // zero displacement: no contribution
            const T inv_r = approx_rsqrt(r2);
            const T q = r2 * inv_r * G.inv_h;
            const T inv_q = G.h * inv_r;
            const T F = kernel_f(G, q, inv_q);
            if (MODE == 4) {
                const T dx = va.x - vb->x, dy = va.y - vb->y, dz = va.z - vb->z;  // lambda_A_a - lambda_A_b
                const T dd = d[0] * dx + d[1] * dy + d[2] * dz;
                de -= Ph.m_g * F * dd;
                const T c = -Ph.m_g * (qa + pb.w);
                const T Fr = kernel_fprime(G, q, inv_q) * inv_r;
                ax += c * (F * dx + Fr * dd * d[0]);
                ay += c * (F * dy + Fr * dd * d[1]);
                az += c * (F * dz + Fr * dd * d[2]);
            } else {
                const T c = Ph.m_g * F * (rhoa + rhob);
                ax += c * d[0];
                ay += c * d[1];
                az += c * d[2];
            }
            return;
        }
        if (MODE <= 1) {
            sum += kernel_w(G, approx_sqrt(r2) * G.inv_h);
            if (MODE == 1) {
                ++cnt;
                fp += (uint64_t)((idb & kIdMask) + 1u) * 0x9E3779B97F4A7C15ull;
            }
        } else {
            if (r2 == T(0)) return;  // self or coincident particle: zero gradient
            const T inv_r = approx_rsqrt(r2);
            const T F = kernel_f(G, r2 * inv_r * G.inv_h, G.h * inv_r);  // (1/r) dW/dr
            T coef = qa + pb.w;
            if (MODE == 3) {
                const T vx = va.x - vb->x, vy = va.y - vb->y, vz = va.z - vb->z;
                const T vr = vx * d[0] + vy * d[1] + vz * d[2];
                T pi = T(0);
                if (Ph.av && vr < T(0)) {
                    const T mu = approx_div(Ph.h * vr, r2 + Ph.eta2);
                    const T cb = Ph.eos == TFSPH_EOS_ADIABATIC ? approx_sqrt(Ph.gamma * Ph.gm1 * vb->w) : Ph.cs;
                    const T cbar = T(0.5) * (ca + cb);
                    const T rbar = T(0.5) * (rhoa + rhob);
                    pi = approx_div(-Ph.av_alpha * cbar * mu + Ph.av_beta * mu * mu, rbar);
                }
                coef += pi;
                de += (qa + T(0.5) * pi) * vr * F;
            }
            const T s = coef * F;
            ax -= s * d[0];
            ay -= s * d[1];
            az -= s * d[2];
        }
    }
};

// Loads the per-particle data of particle a and prepares the accumulator.
template <class T, int MODE>
__device__ __forceinline__ void acc_init(PairAcc<T, MODE> &A, const Phys<T> &Ph, const V4<T> &pa,
                                         const V4<T> *__restrict__ vel, const T *__restrict__ rho, uint32_t a)
{
    if (MODE == 4) {
        A.qa = pa.w;
        A.va = vel[a];  // lambda_A_a
        return;
    }
    if (MODE == 5) {
        A.rhoa = rho[a];  // lambda_rho_a
        return;
    }
    if (MODE >= 2) {
        A.qa = pa.w;
        A.ca = Ph.cs;
        if (MODE == 3) {
            A.va = vel[a];
            A.rhoa = rho[a];
            if (Ph.eos == TFSPH_EOS_ADIABATIC) A.ca = sqrt(Ph.gamma * Ph.gm1 * A.va.w);
        }
    }
}

template <class T, int MODE>
__device__ __forceinline__ void acc_store(const PairAcc<T, MODE> &A, const Phys<T> &Ph, uint32_t a, T mass,
                                          const V4<T> *__restrict__ vel, T *__restrict__ out_rho, T *pr_out,
                                          V4<T> *__restrict__ out_acc, int32_t *__restrict__ cnt,
                                          uint64_t *__restrict__ fpr)
{
    if (MODE == 4) {
        // lambda_rho_a = dq/drho lambda_q_a = -cs^2/rho^2 lambda_q_a (isothermal q = cs^2/rho)
        const T ra = vel == nullptr ? T(1) : out_rho[a];
        (void)ra;
        V4<T> o;
        o.x = A.ax;
        o.y = A.ay;
        o.z = A.az;
        o.w = A.de;  // lambda_q_a, turned into lambda_rho by the caller
        out_acc[a] = o;
        return;
    }
    if (MODE == 5) {
        V4<T> o = out_acc[a];
        o.x += A.ax;
        o.y += A.ay;
        o.z += A.az;
        out_acc[a] = o;
        return;
    }
    if (MODE <= 1) {
        const T r = mass * A.sum;
        out_rho[a] = r;
        if (pr_out) {
            const T pr = Ph.eos == TFSPH_EOS_ADIABATIC ? Ph.gm1 * vel[a].w / r : Ph.cs2 / r;
            pr_out[4 * (size_t)a + 3] = pr;  // .w of pos[a]; the other lanes are untouched
        }
        if (MODE == 1) {
            cnt[a] = A.cnt;
            fpr[a] = A.fp;
        }
    } else {
        V4<T> o;
        o.x = Ph.m_g * A.ax;
        o.y = Ph.m_g * A.ay;
        o.z = Ph.m_g * A.az;
        o.w = Ph.m_g * A.de;
        out_acc[a] = o;
    }
}

// ---------------------------------------------------------------------------
// Global-memory candidate walk (fallback, and axes whose window wraps fully)
// ---------------------------------------------------------------------------
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

// Largest offsets (ohi >= 0, olo <= 0) along x whose cell slab lies within the
// squared radius rem of a particle at fractional position fx.
template <class T>
__device__ __forceinline__ void x_window(const Geo<T> &G, T fx, T rem, int &olo, int &ohi)
{
    ohi = 0;
    olo = 0;
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
}

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
                int olo, ohi;
                x_window(G, fx, G.lim2 - dz2 - dy2, olo, ohi);
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

template <class T, int DIM, int MODE>
__device__ __forceinline__ void walk_global(PairAcc<T, MODE> &A, const Geo<T> &G, const Phys<T> &Ph,
                                            const V4<T> &pa, const V4<T> *__restrict__ pos,
                                            const V4<T> *__restrict__ vel, const T *__restrict__ rho,
                                            const uint32_t *__restrict__ id, const uint32_t *__restrict__ start)
{
    for_each_row<T, DIM>(G, start, pa.x, pa.y, pa.z, [&](const RowRanges &rr) {
        const uint32_t tot = rr.total();
        for (uint32_t i = 0; i < tot; ++i) {
            const uint32_t b = rr.at(i);
            const V4<T> pb = pos[b];
            T d[3];
            const T r2 = pair_r2<T, DIM, true>(G, pa, pb, d);
            V4<T> vb;
            T rhob = T(1);
            if (r2 < G.h2x4) {
                if (ModeUses<MODE>::vel) vb = vel[b];
                if (ModeUses<MODE>::rho) rhob = rho[b];
            }
            A.add(G, Ph, pb, &vb, rhob, MODE == 1 ? id[b] : 0u, r2, d);
        }
    });
}

// One thread per particle, candidates from global memory.
template <class T, int DIM, int MODE>
__global__ void __launch_bounds__(128, 1)
k_pair_global(Geo<T> G, Phys<T> Ph, const V4<T> *__restrict__ pos, const V4<T> *__restrict__ vel,
              const T *__restrict__ rho, const uint32_t *__restrict__ id, const uint32_t *__restrict__ start, int n,
              T mass, T *__restrict__ out_rho, T *pr_out, V4<T> *__restrict__ out_acc, int32_t *__restrict__ cnt,
              uint64_t *__restrict__ fpr)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const V4<T> pa = pos[a];
    PairAcc<T, MODE> A;
    acc_init(A, Ph, pa, vel, rho, a);
    walk_global<T, DIM, MODE>(A, G, Ph, pa, pos, vel, rho, id, start);
    acc_store(A, Ph, a, mass, vel, out_rho, pr_out, out_acc, cnt, fpr);
}

// ---------------------------------------------------------------------------
// Tiled path
// ---------------------------------------------------------------------------
struct TileCfg {
    int T[3];     // owned cells per axis
    int H[3];     // halo cells per axis (T + 2R)
    int nt[3];    // tiles per axis
    int nhalo;    // H0 H1 H2
    int nrows;    // T1 T2 owned rows
    int cap;      // particles that fit in shared memory
    int offset;   // byte offset of the particle arrays in shared memory
    float invH[2];  // 1 / H0, 1 / H1
};

// q = floor(x / d) for 0 <= x < 2^22 and 0 < d < 2^10 by a float multiply with
// the rounded reciprocal: (x + 1/2)/d lies at least 1/(2d) from an integer,
// more than the product's rounding error, so the truncation is exact.
__device__ __forceinline__ int small_div(int x, int d, float inv_d)
{
    return (int)(((float)x + 0.5f) * inv_d);
}

// Halo cell h -> (hx, hy, hz), without integer division.
__device__ __forceinline__ void halo_coords(int h, const TileCfg &C, int &hx, int &hy, int &hz)
{
    const int row = small_div(h, C.H[0], C.invH[0]);
    hx = h - row * C.H[0];
    hz = small_div(row, C.H[1], C.invH[1]);
    hy = row - hz * C.H[1];
}

// In-place exclusive scan of m values in shared memory by the whole block;
// a[m] receives the total.
__device__ void block_scan_smem(int *a, int m, int *wsum)
{
    const int tid = threadIdx.x, nth = blockDim.x;
    const int chunk = (m + nth - 1) / nth;
    const int b0 = min(m, tid * chunk), b1 = min(m, b0 + chunk);
    int s = 0;
    for (int i = b0; i < b1; ++i) s += a[i];
    const int lane = tid & 31, wid = tid >> 5;
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < (nth >> 5) ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < (nth >> 5)) wsum[lane] = t;
    }
    __syncthreads();
    int run = (wid > 0 ? wsum[wid - 1] : 0) + x - s;
    for (int i = b0; i < b1; ++i) {
        const int v = a[i];
        a[i] = run;
        run += v;
    }
    if (tid == nth - 1) a[m] = run;
    __syncthreads();
}

// Global cell coordinate of halo coordinate hc along axis k (-1: none).
template <class T>
__device__ __forceinline__ int halo_cell(const Geo<T> &G, int k, int c0, int hc)
{
    return axis_wrap(c0 - G.R[k] + hc, G.n[k], G.per[k]);
}

// 1 if halo coordinate hc along axis k lies across the periodic seam.
template <class T>
__device__ __forceinline__ int halo_seam(const Geo<T> &G, int k, int c0, int hc)
{
    const int g = c0 - G.R[k] + hc;
    return G.per[k] && (g < 0 || g >= G.n[k]);
}

template <class T, int DIM, int MODE, bool SEAM>
__device__ __forceinline__ void walk_smem_range(PairAcc<T, MODE> &A, const Geo<T> &G, const Phys<T> &Ph,
                                                const V4<T> &pa, const V4<T> *spos, const V4<T> *svel,
                                                const T *srho, const uint32_t *sid, int j0, int j1)
{
    for (int j = j0; j < j1; ++j) {
        const V4<T> pb = spos[j];
        T d[3];
        const T r2 = pair_r2<T, DIM, SEAM>(G, pa, pb, d);
        if (ModeUses<MODE>::vel || ModeUses<MODE>::rho) {
            if (r2 < G.h2x4)
                A.add(G, Ph, pb, ModeUses<MODE>::vel ? &svel[j] : nullptr, ModeUses<MODE>::rho ? srho[j] : T(1), 0u,
                      r2, d);
        } else {
            A.add(G, Ph, pb, nullptr, T(1), MODE == 1 ? sid[j] : 0u, r2, d);
        }
    }
}

// Candidate walk of one owned particle over the staged tile.
template <class T, int DIM, int MODE>
__device__ __forceinline__ void walk_tile(PairAcc<T, MODE> &A, const Geo<T> &G, const Phys<T> &Ph, const TileCfg &C,
                                          const int c0[3], const V4<T> &pa, const int *lstart, const V4<T> *spos,
                                          const V4<T> *svel, const T *srho, const uint32_t *sid)
{
    T tx_, ty_ = T(0), tz_ = T(0);
    const int cx = axis_cell(pa.x, G.lo[0], G.inv_w[0], G.n[0], tx_);
    const int cy = DIM > 1 ? axis_cell(pa.y, G.lo[1], G.inv_w[1], G.n[1], ty_) : 0;
    const int cz = DIM > 2 ? axis_cell(pa.z, G.lo[2], G.inv_w[2], G.n[2], tz_) : 0;
    const T fx = tx_ - T(cx);
    const T fy = DIM > 1 ? ty_ - T(cy) : T(0);
    const T fz = DIM > 2 ? tz_ - T(cz) : T(0);
    const int hx = cx - c0[0] + G.R[0];
    const int hy = DIM > 1 ? cy - c0[1] + G.R[1] : 0;
    const int hz = DIM > 2 ? cz - c0[2] + G.R[2] : 0;
    // x seam bounds in halo coordinates: cells below sx0 or from sx1 on lie across
    const int sx0 = G.per[0] ? G.R[0] - c0[0] : -1;
    const int sx1 = G.per[0] ? G.n[0] - c0[0] + G.R[0] : C.H[0] + 1;
    const int Rz = DIM > 2 ? G.R[2] : 0;
    const int Ry = DIM > 1 ? G.R[1] : 0;
#pragma unroll 1
    for (int oz = -Rz; oz <= Rz; ++oz) {
        T dz2 = T(0);
        int seam_z = 0;
        if (DIM > 2) {
            const T s = slab_dist(oz, fz) * G.w[2];
            dz2 = s * s;
            if (dz2 >= G.lim2) continue;
            seam_z = halo_seam(G, 2, c0[2], hz + oz);
        }
#pragma unroll 1
        for (int oy = -Ry; oy <= Ry; ++oy) {
            T dy2 = T(0);
            int seam_y = 0;
            if (DIM > 1) {
                const T s = slab_dist(oy, fy) * G.w[1];
                dy2 = s * s;
                if (dz2 + dy2 >= G.lim2) continue;
                seam_y = halo_seam(G, 1, c0[1], hy + oy);
            }
            // x window: the cells whose slab lies within t = sqrt(rem)/w of the
            // particle, (o - fx) <= t for o > 0 and (fx + |o| - 1) <= t for o < 0
            const T t = approx_sqrt(G.lim2 - dz2 - dy2) * G.inv_w[0];
            const int ohi = min(G.R[0], max(0, (int)floor(fx + t)));
            const int olo = -min(G.R[0], max(0, (int)floor(t - fx + T(1))));
            const int hrow = C.H[0] * ((hy + oy) + C.H[1] * (hz + oz));
            const int u0 = hx + olo, u1 = hx + ohi + 1;  // halo x cells [u0, u1)
            // [u0, a0) across the low seam, [a0, a1) inside, [a1, u1) across the high seam
            const int a0 = min(max(u0, sx0), u1);
            const int a1 = max(min(u1, sx1), a0);
            const bool inner_seam = (seam_y | seam_z) != 0;
            if (!inner_seam && a1 > a0)
                walk_smem_range<T, DIM, MODE, false>(A, G, Ph, pa, spos, svel, srho, sid, lstart[hrow + a0],
                                                     lstart[hrow + a1]);
            if (inner_seam || a0 > u0 || u1 > a1) {
                // the rare ranges across a seam, visited with the two-sum displacement
                const int j0 = lstart[hrow + (inner_seam ? u0 : (a0 > u0 ? u0 : a1))];
                const int j1 = lstart[hrow + (inner_seam ? u1 : (u1 > a1 ? u1 : a0))];
                const int jm0 = (!inner_seam && a0 > u0 && u1 > a1) ? lstart[hrow + a0] : j1;
                const int jm1 = (!inner_seam && a0 > u0 && u1 > a1) ? lstart[hrow + a1] : j1;
                // [j0, jm0) and [jm1, j1): the inner part [jm0, jm1) was visited above
                for (int j = j0; j < j1; ++j) {
                    if (j == jm0) j = jm1;
                    if (j >= j1) break;
                    walk_smem_range<T, DIM, MODE, true>(A, G, Ph, pa, spos, svel, srho, sid, j, j + 1);
                }
            }
        }
    }
}

template <class T, int DIM, int MODE>
__global__ void __launch_bounds__(kTileThreads, sizeof(T) == 4 ? 3 : 1)
k_pair_tile(Geo<T> G, Phys<T> Ph, TileCfg C, const V4<T> *__restrict__ pos, const V4<T> *__restrict__ vel,
            const T *__restrict__ rho, const uint32_t *__restrict__ id, const uint32_t *__restrict__ start, T mass,
            T *__restrict__ out_rho, T *pr_out, V4<T> *__restrict__ out_acc, int32_t *__restrict__ cnt,
            uint64_t *__restrict__ fpr)
{
    extern __shared__ __align__(64) unsigned char smem[];
    __shared__ int wsum[kTileThreads / 32];
    int *lstart = reinterpret_cast<int *>(smem);      // nhalo + 1
    int *rowpref = lstart + C.nhalo + 1;               // nrows + 1
    int *rowg = rowpref + C.nrows + 1;                 // nrows
    V4<T> *spos = reinterpret_cast<V4<T> *>(smem + C.offset);
    V4<T> *svel = spos + C.cap;                        // modes staging a second V4
    T *srho = reinterpret_cast<T *>(svel + (ModeUses<MODE>::vel ? C.cap : 0));  // modes staging a scalar
    uint32_t *sid = reinterpret_cast<uint32_t *>(spos + C.cap);  // MODE 1

    const int tid = threadIdx.x;
    int b = blockIdx.x;
    const int tx = b % C.nt[0];
    b /= C.nt[0];
    const int ty = b % C.nt[1];
    const int tz = b / C.nt[1];
    const int c0[3] = {tx * C.T[0], ty * C.T[1], tz * C.T[2]};
    int ext[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) ext[k] = min(C.T[k], G.n[k] - c0[k]);

    // owned rows: global start and particle count
    for (int r = tid; r < C.nrows; r += blockDim.x) {
        const int oy = r % C.T[1], oz = r / C.T[1];
        int c = 0, g = 0;
        if (oy < ext[1] && oz < ext[2]) {
            const uint32_t rowkey =
                (uint32_t)G.n[0] * ((uint32_t)(c0[1] + oy) + (uint32_t)G.n[1] * (uint32_t)(c0[2] + oz));
            g = (int)start[rowkey + c0[0]];
            c = (int)start[rowkey + c0[0] + ext[0]] - g;
        }
        rowg[r] = g;
        rowpref[r] = c;
    }
    // halo cell counts; a ragged tile needs only ext + 2R halo cells per axis,
    // which keeps every raw coordinate within (-n, 2n) so one wrap suffices
    for (int h = tid; h < C.nhalo; h += blockDim.x) {
        int hx, hy, hz;
        halo_coords(h, C, hx, hy, hz);
        const bool inside = hx < ext[0] + 2 * G.R[0] && hy < ext[1] + 2 * G.R[1] && hz < ext[2] + 2 * G.R[2];
        const int gx = inside ? halo_cell(G, 0, c0[0], hx) : -1;
        const int gy = DIM > 1 ? halo_cell(G, 1, c0[1], hy) : 0;
        const int gz = DIM > 2 ? halo_cell(G, 2, c0[2], hz) : 0;
        int c = 0;
        if (gx >= 0 && gy >= 0 && gz >= 0) {
            const uint32_t key = (uint32_t)gx + (uint32_t)G.n[0] * ((uint32_t)gy + (uint32_t)G.n[1] * (uint32_t)gz);
            c = (int)(start[key + 1] - start[key]);
        }
        lstart[h] = c;
    }
    __syncthreads();
    block_scan_smem(lstart, C.nhalo, wsum);
    block_scan_smem(rowpref, C.nrows, wsum);
    const int total = lstart[C.nhalo];
    const int owned = rowpref[C.nrows];
    const bool tiled = total <= C.cap;

    if (tiled) {
        for (int h = tid; h < C.nhalo; h += blockDim.x) {
            const int j0 = lstart[h], j1 = lstart[h + 1];
            if (j1 == j0) continue;
            int hx, hy, hz;
            halo_coords(h, C, hx, hy, hz);
            const int gx = halo_cell(G, 0, c0[0], hx);
            const int gy = DIM > 1 ? halo_cell(G, 1, c0[1], hy) : 0;
            const int gz = DIM > 2 ? halo_cell(G, 2, c0[2], hz) : 0;
            const uint32_t key = (uint32_t)gx + (uint32_t)G.n[0] * ((uint32_t)gy + (uint32_t)G.n[1] * (uint32_t)gz);
            const uint32_t g0 = start[key];
            for (int j = j0; j < j1; ++j) {
                const uint32_t gi = g0 + (uint32_t)(j - j0);
                spos[j] = pos[gi];
                if (ModeUses<MODE>::vel) svel[j] = vel[gi];
                if (ModeUses<MODE>::rho) srho[j] = rho[gi];
                if (MODE == 1) sid[j] = id[gi];
            }
        }
        __syncthreads();
    }

    for (int p = tid; p < owned; p += blockDim.x) {
        // owned row of p: the last r with rowpref[r] <= p
        int lo = 0, hi = C.nrows - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (rowpref[mid] <= p) lo = mid; else hi = mid - 1;
        }
        const int k = p - rowpref[lo];
        const uint32_t a = (uint32_t)(rowg[lo] + k);
        PairAcc<T, MODE> A;
        if (!tiled) {
            const V4<T> pa = pos[a];
            acc_init(A, Ph, pa, vel, rho, a);
            walk_global<T, DIM, MODE>(A, G, Ph, pa, pos, vel, rho, id, start);
        } else {
            // the owned row starts at halo x = R of halo row (oy + R, oz + R)
            const int oy = lo % C.T[1], oz = lo / C.T[1];
            const int hrow = C.H[0] * ((oy + (DIM > 1 ? G.R[1] : 0)) + C.H[1] * (oz + (DIM > 2 ? G.R[2] : 0)));
            const V4<T> pa = spos[lstart[hrow + G.R[0]] + k];
            acc_init(A, Ph, pa, vel, rho, a);
            walk_tile<T, DIM, MODE>(A, G, Ph, C, c0, pa, lstart, spos, svel, srho, sid);
        }
        acc_store(A, Ph, a, mass, vel, out_rho, pr_out, out_acc, cnt, fpr);
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <class T, int MODE> constexpr int tile_bytes_per_particle()
{
    return (int)sizeof(V4<T>) + (ModeUses<MODE>::vel ? (int)sizeof(V4<T>) : 0) +
           (ModeUses<MODE>::rho ? (int)sizeof(T) : 0) + (MODE == 1 ? 4 : 0);
}

// Tile shape for a phase with `mean` particles per cell. Each CTA thread
// takes one owned particle, so a tile is sized to hold about 7/8 of the
// block's threads on average (a tile holding more than one particle per
// thread runs a second, mostly idle pass); its halo must fill at most 80 %
// of the shared-memory capacity. Returns false when an axis wraps fully.
template <class T>
bool plan_tiles(const Geo<T> &G, int dim, double mean, int bytes_pp, int smem_budget, TileCfg &C, size_t &smem)
{
    for (int k = 0; k < dim; ++k)
        if (G.full[k]) return false;
    const double target_cells = std::max(1.0, 0.875 * kTileThreads / std::max(mean, 1e-6));
    const int side = std::max(1, (int)std::floor(std::pow(target_cells, 1.0 / dim) + 1e-9));
    int Tt[3] = {1, 1, 1};
    for (int k = 1; k < dim; ++k) Tt[k] = std::min(side, G.n[k]);
    double rest = 1.0;
    for (int k = 1; k < dim; ++k) rest *= Tt[k];
    Tt[0] = std::max(1, std::min(G.n[0], (int)std::floor(target_cells / rest + 1e-9)));
    for (;;) {
        int H[3] = {1, 1, 1};
        long nh = 1;
        for (int k = 0; k < dim; ++k) {
            H[k] = Tt[k] + 2 * G.R[k];
            nh *= H[k];
        }
        const long nrows = (long)Tt[1] * Tt[2];
        const long table = 4 * (nh + 1 + 2 * nrows + 1);
        const long offset = (table + 63) / 64 * 64;
        const long cap = (smem_budget - offset) / bytes_pp;
        const double expected = mean * (double)nh;
        int kmax = 0;
        for (int k = 1; k < dim; ++k)
            if (Tt[k] > Tt[kmax]) kmax = k;
        if ((cap > 0 && expected <= 0.8 * (double)cap) || Tt[kmax] == 1) {
            if (cap <= 0 || nh >= (1L << 22) || H[0] >= 1024 || H[1] >= 1024) return false;
            for (int k = 0; k < 3; ++k) {
                C.T[k] = Tt[k];
                C.H[k] = H[k];
                C.nt[k] = k < dim ? (G.n[k] + Tt[k] - 1) / Tt[k] : 1;
            }
            C.nhalo = (int)nh;
            C.nrows = (int)nrows;
            C.invH[0] = 1.0f / (float)H[0];
            C.invH[1] = 1.0f / (float)H[1];
            C.cap = (int)cap;
            C.offset = (int)offset;
            smem = (size_t)offset + (size_t)cap * (size_t)bytes_pp;
            return true;
        }
        Tt[kmax] = (Tt[kmax] + 1) / 2;
    }
}

template <class T, int DIM, int MODE>
cudaError_t pair_launch(const LaunchCtx &L, const Geo<T> &G, const Phys<T> &Ph, int n, T mass, const V4<T> *pos,
                        const V4<T> *vel, const T *rho, const uint32_t *id, const uint32_t *start, T *out_rho,
                        T *pr_out, V4<T> *out_acc, int32_t *cnt, uint64_t *fpr, double mean)
{
    constexpr int bpp = tile_bytes_per_particle<T, MODE>();
    const int budget = (ModeUses<MODE>::vel || ModeUses<MODE>::rho) ? 72 * 1024 : 52 * 1024;
    TileCfg C{};
    size_t smem = 0;
    if (plan_tiles(G, DIM, mean, bpp, budget, C, smem)) {
        static bool attr_set = false;
        if (!attr_set) {
            cudaError_t e = cudaFuncSetAttribute(k_pair_tile<T, DIM, MODE>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, budget);
            if (e != cudaSuccess) return e;
            attr_set = true;
        }
        const int blocks = C.nt[0] * C.nt[1] * C.nt[2];
        k_pair_tile<T, DIM, MODE><<<blocks, kTileThreads, smem, L.stream>>>(G, Ph, C, pos, vel, rho, id, start, mass,
                                                                            out_rho, pr_out, out_acc, cnt, fpr);
    } else {
        const int threads = 128;
        k_pair_global<T, DIM, MODE><<<(n + threads - 1) / threads, threads, 0, L.stream>>>(
            G, Ph, pos, vel, rho, id, start, n, mass, out_rho, pr_out, out_acc, cnt, fpr);
    }
    return cudaGetLastError();
}

template <class T, int DIM>
cudaError_t density_t(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &P, void *rho, bool gas,
                      int32_t *cnt, uint64_t *fprint)
{
    if (P.n == 0) return cudaSuccess;
    const Geo<T> &G = *static_cast<const Geo<T> *>(geo);
    const Phys<T> &Ph = *static_cast<const Phys<T> *>(phys);
    auto *pos = static_cast<V4<T> *>(P.pos[P.cur]);
    auto *vel = static_cast<const V4<T> *>(P.vel[P.cur]);
    T *pr = gas ? reinterpret_cast<T *>(pos) : nullptr;
    const T mass = gas ? Ph.m_g : Ph.m_d;
    const double mean = (double)P.n / (double)G.ncells;
    if (cnt)
        return pair_launch<T, DIM, 1>(L, G, Ph, (int)P.n, mass, pos, vel, nullptr, P.id[P.cur], P.start,
                                      static_cast<T *>(rho), pr, nullptr, cnt, fprint, mean);
    return pair_launch<T, DIM, 0>(L, G, Ph, (int)P.n, mass, pos, vel, nullptr, P.id[P.cur], P.start,
                                  static_cast<T *>(rho), pr, nullptr, nullptr, nullptr, mean);
}

template <class T, int DIM>
cudaError_t force_t(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &P, const void *rho, void *acc)
{
    if (P.n == 0) return cudaSuccess;
    const Geo<T> &G = *static_cast<const Geo<T> *>(geo);
    const Phys<T> &Ph = *static_cast<const Phys<T> *>(phys);
    auto *pos = static_cast<const V4<T> *>(P.pos[P.cur]);
    auto *vel = static_cast<const V4<T> *>(P.vel[P.cur]);
    const double mean = (double)P.n / (double)G.ncells;
    const bool full = Ph.av || Ph.eos == TFSPH_EOS_ADIABATIC;
    if (full)
        return pair_launch<T, DIM, 3>(L, G, Ph, (int)P.n, T(0), pos, vel, static_cast<const T *>(rho), P.id[P.cur],
                                      P.start, nullptr, nullptr, static_cast<V4<T> *>(acc), nullptr, nullptr, mean);
    return pair_launch<T, DIM, 2>(L, G, Ph, (int)P.n, T(0), pos, vel, static_cast<const T *>(rho), P.id[P.cur],
                                  P.start, nullptr, nullptr, static_cast<V4<T> *>(acc), nullptr, nullptr, mean);
}

// lambda_A (V4, storage order) -> lambda_x (V4 .xyz) and lambda_q (.w).
template <class T, int DIM>
cudaError_t force_adjoint_t(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &P, const void *lamA,
                            void *out)
{
    if (P.n == 0) return cudaSuccess;
    const Geo<T> &G = *static_cast<const Geo<T> *>(geo);
    const Phys<T> &Ph = *static_cast<const Phys<T> *>(phys);
    auto *pos = static_cast<const V4<T> *>(P.pos[P.cur]);
    const double mean = (double)P.n / (double)G.ncells;
    return pair_launch<T, DIM, 4>(L, G, Ph, (int)P.n, T(0), pos, static_cast<const V4<T> *>(lamA), nullptr,
                                  P.id[P.cur], P.start, nullptr, nullptr, static_cast<V4<T> *>(out), nullptr, nullptr,
                                  mean);
}

// lambda_rho (T, storage order) -> lambda_x (V4 .xyz) accumulated.
template <class T, int DIM>
cudaError_t density_adjoint_t(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &P,
                              const void *lamrho, void *inout)
{
    if (P.n == 0) return cudaSuccess;
    const Geo<T> &G = *static_cast<const Geo<T> *>(geo);
    const Phys<T> &Ph = *static_cast<const Phys<T> *>(phys);
    auto *pos = static_cast<const V4<T> *>(P.pos[P.cur]);
    const double mean = (double)P.n / (double)G.ncells;
    return pair_launch<T, DIM, 5>(L, G, Ph, (int)P.n, T(0), pos, nullptr, static_cast<const T *>(lamrho),
                                  P.id[P.cur], P.start, nullptr, nullptr, static_cast<V4<T> *>(inout), nullptr,
                                  nullptr, mean);
}

}  // namespace

cudaError_t launch_force_adjoint(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G,
                                 const void *lamA, void *out)
{
    if (L.precision == TFSPH_FP64) {
        switch (L.dim) {
            case 1: return force_adjoint_t<double, 1>(L, geo, phys, G, lamA, out);
            case 2: return force_adjoint_t<double, 2>(L, geo, phys, G, lamA, out);
            default: return force_adjoint_t<double, 3>(L, geo, phys, G, lamA, out);
        }
    }
    switch (L.dim) {
        case 1: return force_adjoint_t<float, 1>(L, geo, phys, G, lamA, out);
        case 2: return force_adjoint_t<float, 2>(L, geo, phys, G, lamA, out);
        default: return force_adjoint_t<float, 3>(L, geo, phys, G, lamA, out);
    }
}

cudaError_t launch_density_adjoint(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G,
                                   const void *lamrho, void *inout)
{
    if (L.precision == TFSPH_FP64) {
        switch (L.dim) {
            case 1: return density_adjoint_t<double, 1>(L, geo, phys, G, lamrho, inout);
            case 2: return density_adjoint_t<double, 2>(L, geo, phys, G, lamrho, inout);
            default: return density_adjoint_t<double, 3>(L, geo, phys, G, lamrho, inout);
        }
    }
    switch (L.dim) {
        case 1: return density_adjoint_t<float, 1>(L, geo, phys, G, lamrho, inout);
        case 2: return density_adjoint_t<float, 2>(L, geo, phys, G, lamrho, inout);
        default: return density_adjoint_t<float, 3>(L, geo, phys, G, lamrho, inout);
    }
}

cudaError_t launch_density(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &P, void *rho, bool gas,
                           int32_t *cnt, uint64_t *fprint)
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
