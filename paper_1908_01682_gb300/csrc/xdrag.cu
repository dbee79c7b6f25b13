// The two other drag schemes of the paper on the same binning, densities and
// gas pressure force: ISPH (Sec. 2.2, Eqs. 11-16) and MK (Sec. 2.1,
// Eqs. 8-10).
//
// Drag coefficient K = rho_d / t_stop (Eq. 7) with the per-particle stopping
// times t_j (vel.w of the dust); at a gas particle ISPH interpolates K like
// any dust field: K_a = m_d sum_j W_aj / t_j. In MK, K_aj / (rho_a,g rho_j,d)
// = 1 / (rho_a,g t_j), sigma = the dimension, eta^2 = 0.001 h^2. Frozen
// (wall) gas particles enter the density and pressure sums and take no part
// in the drag.
//
// Cross-phase sums: one thread per target particle walks the other phase's
// candidate cells in global memory (the row walk of the gas pair sums), with
// the same neighbour decision r^2 < 4h^2.
//   ISPH at gas a over dust:  rho^d_a = m_d sum W,  K_a,  u_a = m_d sum u_j/rho_j W
//   ISPH at dust j over gas:  rho^g_j = m_g sum W,  v_j = m_g sum_moving v_a/rho_a W,
//     e_j (adiabatic), pressure acceleration A_j = -(Q_j + q_j G_j) (Eq. 14)
//     with G_j = m_g sum grad_j W, Q_j = m_g sum q_a grad_j W, q_j = p_j/rho_j^2
//   MK at gas a:  D_a = -sigma m_d / rho_a sum_j ((v_a - u_j).d)/(r^2 + eta^2) d W / t_j
//   MK at dust j: D_j =  sigma m_g / t_j sum_a ((v_a - u_j).d)/(r^2 + eta^2) d W / rho_a
// (d = x_target - x_source; ((v_a - u_j).r) r is even in r).
// Then one thread per particle: the ISPH 2x2 implicit solve in (own velocity,
// interpolated velocity of the other phase)
//   w' = (v - u + tau A) / (1 + tau (alpha + beta)),  alpha = K/rho_g, beta = K/rho_d,
//   gas keeps v' = v + tau (A + g) - tau alpha w', dust keeps u' = u + tau g + tau beta w',
// or the MK explicit update v' = v + tau (A + D + g), u' = u + tau (D + g); then
// x' = x + tau v' (periodic wrap) and the next cell keys.
#include "pair.cuh"

namespace tfsph {
namespace {

constexpr int kXThreads = 128;

enum XKind { kIsphAtGas = 0, kIsphAtDust = 1, kMkAtGas = 2, kMkAtDust = 3 };

template <class T> struct XArgs {
    // targets
    const V4<T> *tpos, *tvel;
    const uint32_t *tid;
    const T *trho;      // target density (MK gas: rho_g)
    int n;
    // sources (the other phase)
    const V4<T> *spos, *svel;
    const uint32_t *sid;
    const uint32_t *sstart;
    const T *srho;      // source density (rho_d for ISPH at gas, rho_g otherwise)
    int has_frozen;     // gas carries frozen flags (in tid for gas targets, sid for gas sources)
    // outputs
    V4<T> *out4;        // ISPH gas: (u_a, K_a); ISPH dust: (v_j, rho^g_j); MK: D
    V4<T> *out4b;       // ISPH dust: (A_j, 0)
    T *out1;            // ISPH gas: rho^d_a
};

template <class T, int DIM, int KIND>
__global__ void __launch_bounds__(kXThreads, sizeof(T) == 4 ? 12 : 1) k_xsum(Geo<T> G, Phys<T> Ph, XArgs<T> X)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= X.n) return;
    const bool gas_target = KIND == kIsphAtGas || KIND == kMkAtGas;
    if (gas_target && X.has_frozen && (X.tid[t] & kFrozenBit)) return;
    const V4<T> pt = X.tpos[t];
    const V4<T> vt = X.tvel[t];
    const T eta2 = T(0.001) * G.h * G.h;
    T s0 = T(0), s1 = T(0);                         // rho, K (ISPH gas) / rho, e (ISPH dust)
    T a[3] = {T(0), T(0), T(0)};                    // u_a, v_j or the MK sum
    T gs[3] = {T(0), T(0), T(0)}, qs[3] = {T(0), T(0), T(0)};
    auto range = [&](uint32_t b0, uint32_t n, auto seam) {
        for (uint32_t b = b0; b < b0 + n; ++b) {
            const V4<T> pb = X.spos[b];
            T d[3];
            const T r2 = pair_r2<T, DIM, decltype(seam)::value>(G, pt, pb, d);
            if (!(r2 < G.h2x4)) continue;
            const V4<T> vb = X.svel[b];
            const T r = approx_sqrt(r2);
            const T W = kernel_w(G, r * G.inv_h);
            if (KIND == kIsphAtGas) {
                const T w = Ph.m_d * W;
                s0 += w;
                s1 += approx_div(w, vb.w);  // t_j
                const T c = approx_div(w, X.srho[b]);
                a[0] += c * vb.x;
                a[1] += c * vb.y;
                a[2] += c * vb.z;
            } else if (KIND == kIsphAtDust) {
                const T w = Ph.m_g * W;
                const T inv_rho = approx_div(T(1), X.srho[b]);
                s0 += w;
                if (Ph.eos == TFSPH_EOS_ADIABATIC) s1 += w * vb.w * inv_rho;
                if (!(X.has_frozen && (X.sid[b] & kFrozenBit))) {
                    a[0] += w * vb.x * inv_rho;
                    a[1] += w * vb.y * inv_rho;
                    a[2] += w * vb.z * inv_rho;
                }
                if (r2 > T(0)) {
                    const T F = Ph.m_g * kernel_f(G, r * G.inv_h, approx_div(G.h, r));  // m_g (1/r) dW/dr
                    const T q = pb.w;                                       // p_a / rho_a^2
                    for (int k = 0; k < 3; ++k) {
                        gs[k] += F * d[k];
                        qs[k] += q * F * d[k];
                    }
                }
            } else {
                // MK: ((v_a - u_j) . d) / (r^2 + eta^2) W, times 1/t_j (gas target) or 1/rho_a (dust target)
                if (KIND == kMkAtDust && X.has_frozen && (X.sid[b] & kFrozenBit)) continue;
                T rel;
                if (KIND == kMkAtGas) rel = (vt.x - vb.x) * d[0] + (vt.y - vb.y) * d[1] + (vt.z - vb.z) * d[2];
                else rel = (vb.x - vt.x) * d[0] + (vb.y - vt.y) * d[1] + (vb.z - vt.z) * d[2];
                const T coef = approx_div(T(1), KIND == kMkAtGas ? vb.w : X.srho[b]);
                const T f = approx_div(coef * rel, r2 + eta2) * W;
                a[0] += f * d[0];
                a[1] += f * d[1];
                a[2] += f * d[2];
            }
        }
    };
    for_each_range<T, DIM>(G, X.sstart, pt.x, pt.y, pt.z, [&](uint32_t b0, uint32_t n, bool seam) {
        if (seam) range(b0, n, SeamTag<true>{});
        else range(b0, n, SeamTag<false>{});
    });
    V4<T> o;
    if (KIND == kIsphAtGas) {
        o.x = a[0]; o.y = a[1]; o.z = a[2]; o.w = s1;
        X.out4[t] = o;
        X.out1[t] = s0;
    } else if (KIND == kIsphAtDust) {
        T qj = T(0);
        if (s0 > T(0)) qj = Ph.eos == TFSPH_EOS_ADIABATIC ? Ph.gm1 * s1 / s0 : Ph.cs2 / s0;
        o.x = a[0]; o.y = a[1]; o.z = a[2]; o.w = s0;
        X.out4[t] = o;
        V4<T> A;
        A.x = -(qs[0] + qj * gs[0]);
        A.y = -(qs[1] + qj * gs[1]);
        A.z = -(qs[2] + qj * gs[2]);
        A.w = T(0);
        X.out4b[t] = A;
    } else {
        const T sig = T(DIM);
        const T c = KIND == kMkAtGas ? -sig * Ph.m_d / X.trho[t] : sig * Ph.m_g / vt.w;
        o.x = c * a[0]; o.y = c * a[1]; o.z = c * a[2]; o.w = T(0);
        X.out4[t] = o;
    }
}

// Per-particle updates. SCHEME: TFSPH_DRAG_ISPH or TFSPH_DRAG_MK.
template <class T, int DIM, int SCHEME>
__global__ void __launch_bounds__(256)
k_xupdate_gas(Geo<T> G, Phys<T> Ph, T tau, T g0, T g1, T g2, int has_frozen, V4<T> *__restrict__ pos,
              V4<T> *__restrict__ vel, const uint32_t *__restrict__ id, uint32_t *__restrict__ key,
              const T *__restrict__ rho, const V4<T> *__restrict__ acc, const V4<T> *__restrict__ x4,
              const T *__restrict__ x1, int n)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    V4<T> p = pos[a];
    if (has_frozen && (id[a] & kFrozenBit)) {
        key[a] = cell_key<T, DIM>(G, p.x, p.y, p.z);
        return;
    }
    V4<T> v = vel[a];
    const V4<T> A = acc[a], X = x4[a];
    const T gv[3] = {g0, g1, g2};
    T vv[3] = {v.x, v.y, v.z};
    const T AA[3] = {A.x, A.y, A.z}, XX[3] = {X.x, X.y, X.z};
    if (SCHEME == TFSPH_DRAG_ISPH) {
        const T rd = x1[a];
        if (rd > T(0)) {
            const T alpha = X.w / rho[a], beta = X.w / rd;
            const T den = T(1) + tau * (alpha + beta);
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const T wn = (vv[k] - XX[k] + tau * AA[k]) / den;
                vv[k] = vv[k] + tau * (AA[k] + gv[k]) - tau * alpha * wn;
            }
        } else {
#pragma unroll
            for (int k = 0; k < DIM; ++k) vv[k] = vv[k] + tau * (AA[k] + gv[k]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < DIM; ++k) vv[k] = vv[k] + tau * (AA[k] + XX[k] + gv[k]);
    }
    v.x = vv[0];
    p.x = p.x + tau * vv[0];
    if (G.per[0]) p.x = wrap_periodic(p.x, G.lo[0], G.L[0]);
    if (DIM > 1) {
        v.y = vv[1];
        p.y = p.y + tau * vv[1];
        if (G.per[1]) p.y = wrap_periodic(p.y, G.lo[1], G.L[1]);
    }
    if (DIM > 2) {
        v.z = vv[2];
        p.z = p.z + tau * vv[2];
        if (G.per[2]) p.z = wrap_periodic(p.z, G.lo[2], G.L[2]);
    }
    if (Ph.eos == TFSPH_EOS_ADIABATIC) v.w = v.w + tau * A.w;
    p.w = T(0);
    pos[a] = p;
    vel[a] = v;
    key[a] = cell_key<T, DIM>(G, p.x, p.y, p.z);
}

template <class T, int DIM, int SCHEME>
__global__ void __launch_bounds__(256)
k_xupdate_dust(Geo<T> G, T tau, T g0, T g1, T g2, V4<T> *__restrict__ pos, V4<T> *__restrict__ vel,
               uint32_t *__restrict__ key, const T *__restrict__ rho_d, const V4<T> *__restrict__ x4,
               const V4<T> *__restrict__ x4b, int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    V4<T> p = pos[j];
    V4<T> u = vel[j];
    const V4<T> X = x4[j];
    const T gv[3] = {g0, g1, g2};
    T uu[3] = {u.x, u.y, u.z};
    const T XX[3] = {X.x, X.y, X.z};
    if (SCHEME == TFSPH_DRAG_ISPH) {
        if (X.w > T(0)) {
            const V4<T> A = x4b[j];
            const T AA[3] = {A.x, A.y, A.z};
            const T alpha = rho_d[j] / (X.w * u.w), beta = T(1) / u.w;
            const T den = T(1) + tau * (alpha + beta);
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const T wn = (XX[k] - uu[k] + tau * AA[k]) / den;
                uu[k] = uu[k] + tau * gv[k] + tau * beta * wn;
            }
        } else {
#pragma unroll
            for (int k = 0; k < DIM; ++k) uu[k] = uu[k] + tau * gv[k];
        }
    } else {
#pragma unroll
        for (int k = 0; k < DIM; ++k) uu[k] = uu[k] + tau * (XX[k] + gv[k]);
    }
    u.x = uu[0];
    p.x = p.x + tau * uu[0];
    if (G.per[0]) p.x = wrap_periodic(p.x, G.lo[0], G.L[0]);
    if (DIM > 1) {
        u.y = uu[1];
        p.y = p.y + tau * uu[1];
        if (G.per[1]) p.y = wrap_periodic(p.y, G.lo[1], G.L[1]);
    }
    if (DIM > 2) {
        u.z = uu[2];
        p.z = p.z + tau * uu[2];
        if (G.per[2]) p.z = wrap_periodic(p.z, G.lo[2], G.L[2]);
    }
    pos[j] = p;
    vel[j] = u;
    key[j] = cell_key<T, DIM>(G, p.x, p.y, p.z);
}

unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

template <class T, int DIM>
cudaError_t xdrag_t(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &Gp, PhaseBufs &Dp,
                    const void *rho_g, const void *rho_d, const void *acc, const XDragBufs &B, const StepArgs &S,
                    int scheme)
{
    const Geo<T> &G = *static_cast<const Geo<T> *>(geo);
    const Phys<T> &Ph = *static_cast<const Phys<T> *>(phys);
    const int ng = (int)Gp.n, nd = (int)Dp.n;
    auto *gpos = static_cast<V4<T> *>(Gp.pos[Gp.cur]);
    auto *gvel = static_cast<V4<T> *>(Gp.vel[Gp.cur]);
    auto *dpos = static_cast<V4<T> *>(Dp.pos[Dp.cur]);
    auto *dvel = static_cast<V4<T> *>(Dp.vel[Dp.cur]);
    const T *rg = static_cast<const T *>(rho_g);
    const T *rd = static_cast<const T *>(rho_d);
    XArgs<T> at_gas{gpos, gvel, Gp.id[Gp.cur], rg, ng, dpos, dvel, Dp.id[Dp.cur], Dp.start, rd, S.has_frozen,
                    static_cast<V4<T> *>(B.g4), nullptr, static_cast<T *>(B.g1)};
    XArgs<T> at_dust{dpos, dvel, Dp.id[Dp.cur], rd, nd, gpos, gvel, Gp.id[Gp.cur], Gp.start, rg, S.has_frozen,
                     static_cast<V4<T> *>(B.d4), static_cast<V4<T> *>(B.d4b), nullptr};
    const bool isph = scheme == TFSPH_DRAG_ISPH;
    if (ng > 0) {
        if (isph) k_xsum<T, DIM, kIsphAtGas><<<blocks_for(ng, kXThreads), kXThreads, 0, L.stream>>>(G, Ph, at_gas);
        else k_xsum<T, DIM, kMkAtGas><<<blocks_for(ng, kXThreads), kXThreads, 0, L.stream>>>(G, Ph, at_gas);
    }
    if (nd > 0) {
        if (isph) k_xsum<T, DIM, kIsphAtDust><<<blocks_for(nd, kXThreads), kXThreads, 0, L.stream>>>(G, Ph, at_dust);
        else k_xsum<T, DIM, kMkAtDust><<<blocks_for(nd, kXThreads), kXThreads, 0, L.stream>>>(G, Ph, at_dust);
    }
    const T tau = T(S.tau), g0 = T(S.g[0]), g1 = T(S.g[1]), g2 = T(S.g[2]);
    if (ng > 0) {
        if (isph)
            k_xupdate_gas<T, DIM, TFSPH_DRAG_ISPH><<<blocks_for(ng, 256), 256, 0, L.stream>>>(
                G, Ph, tau, g0, g1, g2, S.has_frozen, gpos, gvel, Gp.id[Gp.cur], Gp.key, rg,
                static_cast<const V4<T> *>(acc), static_cast<const V4<T> *>(B.g4), static_cast<const T *>(B.g1), ng);
        else
            k_xupdate_gas<T, DIM, TFSPH_DRAG_MK><<<blocks_for(ng, 256), 256, 0, L.stream>>>(
                G, Ph, tau, g0, g1, g2, S.has_frozen, gpos, gvel, Gp.id[Gp.cur], Gp.key, rg,
                static_cast<const V4<T> *>(acc), static_cast<const V4<T> *>(B.g4), static_cast<const T *>(B.g1), ng);
    }
    if (nd > 0) {
        if (isph)
            k_xupdate_dust<T, DIM, TFSPH_DRAG_ISPH><<<blocks_for(nd, 256), 256, 0, L.stream>>>(
                G, tau, g0, g1, g2, dpos, dvel, Dp.key, rd, static_cast<const V4<T> *>(B.d4),
                static_cast<const V4<T> *>(B.d4b), nd);
        else
            k_xupdate_dust<T, DIM, TFSPH_DRAG_MK><<<blocks_for(nd, 256), 256, 0, L.stream>>>(
                G, tau, g0, g1, g2, dpos, dvel, Dp.key, rd, static_cast<const V4<T> *>(B.d4),
                static_cast<const V4<T> *>(B.d4b), nd);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_xdrag(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G, PhaseBufs &D,
                         const void *rho_g, const void *rho_d, const void *acc, const XDragBufs &B,
                         const StepArgs &S, int scheme)
{
    if (L.precision == TFSPH_FP64) {
        switch (L.dim) {
            case 1: return xdrag_t<double, 1>(L, geo, phys, G, D, rho_g, rho_d, acc, B, S, scheme);
            case 2: return xdrag_t<double, 2>(L, geo, phys, G, D, rho_g, rho_d, acc, B, S, scheme);
            default: return xdrag_t<double, 3>(L, geo, phys, G, D, rho_g, rho_d, acc, B, S, scheme);
        }
    }
    switch (L.dim) {
        case 1: return xdrag_t<float, 1>(L, geo, phys, G, D, rho_g, rho_d, acc, B, S, scheme);
        case 2: return xdrag_t<float, 2>(L, geo, phys, G, D, rho_g, rho_d, acc, B, S, scheme);
        default: return xdrag_t<float, 3>(L, geo, phys, G, D, rho_g, rho_d, acc, B, S, scheme);
    }
}

}  // namespace tfsph
