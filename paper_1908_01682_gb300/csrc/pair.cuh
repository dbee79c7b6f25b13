// Pair machinery shared by the single-context pair kernels and the batched
// step: the neighbour decision r^2 < 4h^2 in explicitly rounded arithmetic,
// the per-pair work of every pair mode (density, force, their adjoints) and
// the candidate walk over cell rows in global memory.
#pragma once

#include "tfsph_internal.cuh"

namespace tfsph {

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
    // squared distance r2 and displacement d = x_a - x_b (LISTED: b comes from
    // the neighbour list, whose entries passed the same r2 < 4h^2 test)
    template <bool LISTED = false>
    __device__ __forceinline__ void add(const Geo<T> &G, const Phys<T> &Ph, const V4<T> &pb, const V4<T> *vb,
                                        T rhob, uint32_t idb, T r2, const T d[3])
    {
        if (!LISTED && !(r2 < G.h2x4)) return;
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
            sum += kernel_w4(pair_sqrt(r2) * G.inv_h);
            if (MODE == 1) {
                ++cnt;
                fp += (uint64_t)((idb & kIdMask) + 1u) * 0x9E3779B97F4A7C15ull;
            }
        } else if (MODE == 2) {
            // isothermal pressure term; (1/r) dW/dr without its factor fnorm,
            // which acc_store applies once together with m_g
            // self or coincident particle (r^2 below the smallest normal):
            // 1/r taken as 0, so q = 0, g is finite and s d = 0 (no branch)
            const T inv_r = r2 >= pair_r2_min<T>() ? pair_rsqrt(r2) : T(0);
            const T q = r2 * inv_r * G.inv_h;
            const T a = fmax(T(2) - q, T(0));
            const T g = q < T(1) ? T(-3) + T(2.25) * q : (a * a) * (Ph.hm075 * inv_r);
            const T s = (qa + pb.w) * g;
            ax -= s * d[0];
            ay -= s * d[1];
            az -= s * d[2];
        } else {
            if (!(r2 >= pair_r2_min<T>())) return;  // self or coincident particle: zero gradient
            const T inv_r = pair_rsqrt(r2);
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
        const T r = (mass * Ph.wnorm4) * A.sum;
        out_rho[a] = r;
        if (pr_out) {
            const T pr = Ph.eos == TFSPH_EOS_ADIABATIC ? Ph.gm1 * vel[a].w / r : Ph.cs2 / r;
            pr_out[4 * (size_t)a + 3] = pr;  // .w of pos[a]; the other lanes are untouched
        }
        if (MODE == 1) {
            cnt[a] = A.cnt;
            fpr[a] = A.fp;
        }
    } else if (MODE == 2) {
        V4<T> o;
        o.x = Ph.mfnorm * A.ax;
        o.y = Ph.mfnorm * A.ay;
        o.z = Ph.mfnorm * A.az;
        o.w = T(0);
        out_acc[a] = o;
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
// Compile-time flag for the range bodies of the global walk.
template <bool S> struct SeamTag {
    static constexpr bool value = S;
};

// floor(x) as an int, in one conversion (x is a small cell offset).
__device__ __forceinline__ int floor_int(float x) { return __float2int_rd(x); }
__device__ __forceinline__ int floor_int(double x) { return __double2int_rd(x); }

// Offsets (ohi >= 0, olo <= 0) along x of the cells whose slab lies within
// the squared radius rem of a particle at fractional position fx (the
// closed form of the tile walk's x window; at most one cell wider than the
// exact slab test at its ends).
template <class T>
__device__ __forceinline__ void x_window(const Geo<T> &G, T fx, T rem, int &olo, int &ohi)
{
    const T t = approx_sqrt(fmax(rem, T(0))) * G.inv_w[0];
    ohi = min(G.R[0], max(0, floor_int(fx + t)));
    olo = -min(G.R[0], max(0, floor_int(t - fx + T(1))));
}

// Calls f(b, n, seam) for every contiguous storage range [b, b + n) of cells
// that may hold neighbours of a particle at (px, py, pz): per row of cells
// (fixed y, z), the part of its x window wrapped below 0, the part wrapped
// above n - 1, then the main part. seam is true when the range lies across a
// periodic seam from the particle, so its displacements need the periodic
// image; within the particle's own image the plain difference is exact.
template <class T, int DIM, class F>
__device__ __forceinline__ void for_each_range(const Geo<T> &G, const uint32_t *__restrict__ start,
                                               T px, T py, T pz, F &&f)
{
    T tx, ty = T(0), tz = T(0);
    const int cx = axis_cell(px, G.lo[0], G.inv_w[0], G.n[0], tx);
    const int cy = DIM > 1 ? axis_cell(py, G.lo[1], G.inv_w[1], G.n[1], ty) : 0;
    const int cz = DIM > 2 ? axis_cell(pz, G.lo[2], G.inv_w[2], G.n[2], tz) : 0;
    const T fx = tx - T(cx);
    const T fy = DIM > 1 ? ty - T(cy) : T(0);
    const T fz = DIM > 2 ? tz - T(cz) : T(0);

    // offsets bounded like the x window (the slab tests below still decide
    // every row); an axis whose window wraps is scanned in full
    int zlo = 0, zhi = 0;
    if (DIM > 2) {
        if (G.full[2]) {
            zhi = G.n[2] - 1;
        } else {
            const T t = approx_sqrt(G.lim2) * G.inv_w[2];
            zhi = min(G.R[2], max(0, floor_int(fz + t)));
            zlo = -min(G.R[2], max(0, floor_int(t - fz + T(1))));
        }
    }
    const int nx = G.n[0];
    // an axis scanned in full (its window wraps) puts every range across a seam
    bool full_seam = false;
#pragma unroll
    for (int k = 0; k < DIM; ++k) full_seam = full_seam || G.full[k];

#pragma unroll 1
    for (int oz = zlo; oz <= zhi; ++oz) {
        int z = 0;
        T dz2 = T(0);
        bool zseam = false;
        if (DIM > 2) {
            if (G.full[2]) {
                z = oz;
            } else {
                z = axis_wrap(cz + oz, G.n[2], G.per[2]);
                if (z < 0) continue;
                zseam = z != cz + oz;
                const T s = slab_dist(oz, fz) * G.w[2];
                dz2 = s * s;
                if (dz2 >= G.lim2) continue;
            }
        }
        int ylo = 0, yhi = 0;
        if (DIM > 1) {
            if (G.full[1]) {
                yhi = G.n[1] - 1;
            } else {
                const T t = approx_sqrt(G.lim2 - dz2) * G.inv_w[1];
                yhi = min(G.R[1], max(0, floor_int(fy + t)));
                ylo = -min(G.R[1], max(0, floor_int(t - fy + T(1))));
            }
        }
#pragma unroll 1
        for (int oy = ylo; oy <= yhi; ++oy) {
            int y = 0;
            T dy2 = T(0);
            bool yseam = false;
            if (DIM > 1) {
                if (G.full[1]) {
                    y = oy;
                } else {
                    y = axis_wrap(cy + oy, G.n[1], G.per[1]);
                    if (y < 0) continue;
                    yseam = y != cy + oy;
                    const T s = slab_dist(oy, fy) * G.w[1];
                    dy2 = s * s;
                    if (dz2 + dy2 >= G.lim2) continue;
                }
            }
            const bool row_seam = full_seam || zseam || yseam;
            const uint32_t row = (uint32_t)nx * ((uint32_t)y + (uint32_t)G.n[1] * (uint32_t)z);
            if (G.full[0]) {
                const uint32_t b = start[row];
                f(b, start[row + nx] - b, row_seam);
            } else {
                int olo, ohi;
                x_window(G, fx, G.lim2 - dz2 - dy2, olo, ohi);
                int x0 = cx + olo, x1 = cx + ohi;
                if (G.per[0]) {
                    if (x0 < 0) {
                        const uint32_t b = start[row + x0 + nx];
                        f(b, start[row + nx] - b, true);
                        x0 = 0;
                    }
                    if (x1 >= nx) {
                        const uint32_t b = start[row];
                        f(b, start[row + (x1 - nx) + 1] - b, true);
                        x1 = nx - 1;
                    }
                } else {
                    if (x0 < 0) x0 = 0;
                    if (x1 >= nx) x1 = nx - 1;
                }
                const uint32_t b = start[row + x0];
                f(b, start[row + x1 + 1] - b, row_seam);
            }
        }
    }
}

template <class T, int DIM, int MODE>
__device__ __forceinline__ void walk_global(PairAcc<T, MODE> &A, const Geo<T> &G, const Phys<T> &Ph,
                                            const V4<T> &pa, const V4<T> *__restrict__ pos,
                                            const V4<T> *__restrict__ vel, const T *__restrict__ rho,
                                            const uint32_t *__restrict__ id, const uint32_t *__restrict__ start)
{
    auto range = [&](uint32_t b0, uint32_t n, auto seam) {
        for (uint32_t b = b0; b < b0 + n; ++b) {
            const V4<T> pb = pos[b];
            T d[3];
            const T r2 = pair_r2<T, DIM, decltype(seam)::value>(G, pa, pb, d);
            V4<T> vb;
            T rhob = T(1);
            if (r2 < G.h2x4) {
                if (ModeUses<MODE>::vel) vb = vel[b];
                if (ModeUses<MODE>::rho) rhob = rho[b];
            }
            A.add(G, Ph, pb, &vb, rhob, MODE == 1 ? id[b] : 0u, r2, d);
        }
    };
    for_each_range<T, DIM>(G, start, pa.x, pa.y, pa.z, [&](uint32_t b0, uint32_t n, bool seam) {
        if (seam) range(b0, n, SeamTag<true>{});
        else range(b0, n, SeamTag<false>{});
    });
}

}  // namespace tfsph
