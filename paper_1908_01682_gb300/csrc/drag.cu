// Implicit drag in cell (Sec. 2.3, Eqs. 17-21) fused with the particle
// update and the next step's cell keys.
//
// One CTA owns kCellsPerCta consecutive cells and, because particles are
// stored in cell order, the contiguous gas and dust ranges of those cells.
//   Phase 1 (thread per cell, accumulator type A): N, L, sum v, sum u,
//     sum A, sum t_j (or sum 1/t_j) in storage order, then
//       eps* = m_d L / (m_g N)                                (Eq. 17)
//       t*   = sum t_j / L   (or L / sum 1/t_j)               (Eq. 18)
//       w    = v_* - u_*                                      (Eq. 21)
//       w'   = (w + tau Abar) / (1 + tau (1 + eps*)/t*)
//       u_*' = u_* + tau g + (tau/t*) w',  v_*' = u_*' + w'
//     which is the cell average of the implicit Eqs. 19-20.
//   Phase 2 (thread per particle, coalesced): the particle equations of
//     Eqs. 19-20 solved for the new velocity, written in the form
//       v_a' = u_*' + (v_a + tau (A_a + g) - u_*') / (1 + tau eps*/t*)
//       u_j' = v_*' + (u_j + tau g - v_*') / (1 + tau/t*)
//     (well conditioned for tau/t* up to 1e6); explicit update in cells with
//     N = 0 or L = 0; e' = e + tau de/dt; x' = x + tau v' (periodic wrap);
//     next cell key.
// The per-cell results live in shared memory only; nothing per cell is
// written to global memory.
#include "drag_ops.cuh"

namespace tfsph {
namespace {

template <class T, class A, int DIM, bool EST>
__global__ void __launch_bounds__(kCellsPerCta, (sizeof(T) == 4 && sizeof(A) == 4) ? 12 : 1)
k_cell_update(Geo<T> G, Phys<T> Ph, A tau, A g0, A g1, A g2, int harmonic, int has_frozen, int adiabatic,
              V4<T> *__restrict__ gpos, V4<T> *__restrict__ gvel, const uint32_t *__restrict__ gid,
              uint32_t *__restrict__ gkey, const uint32_t *__restrict__ gstart, const V4<T> *__restrict__ acc,
              V4<T> *__restrict__ dpos, V4<T> *__restrict__ dvel, uint32_t *__restrict__ dkey,
              const uint32_t *__restrict__ dstart)
{
    __shared__ T s_us[3][kCellsPerCta];
    __shared__ T s_vs[3][kCellsPerCta];
    __shared__ T s_ig[kCellsPerCta];
    __shared__ T s_id[kCellsPerCta];
    __shared__ int s_drag[kCellsPerCta];

    const uint32_t ncells = G.ncells;
    const uint32_t c0 = blockIdx.x * kCellsPerCta;
    const uint32_t c = c0 + threadIdx.x;
    const A gv[3] = {g0, g1, g2};

    // ---- phase 1: per-cell sums and the implicit solve ----
    int drag = 0;
    if (c < ncells) {
        T un[3] = {T(0), T(0), T(0)}, vn[3] = {T(0), T(0), T(0)}, ig = T(0), id = T(0);
        drag = cell_drag_solve<T, A, DIM>(Ph, tau, gv, harmonic, has_frozen, gvel, gid, acc, gstart[c],
                                          gstart[c + 1], dvel, dstart[c], dstart[c + 1], un, vn, ig, id);
        if (drag) {
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                s_us[k][threadIdx.x] = un[k];
                s_vs[k][threadIdx.x] = vn[k];
            }
            s_ig[threadIdx.x] = ig;
            s_id[threadIdx.x] = id;
        }
    }
    s_drag[threadIdx.x] = drag;
    __syncthreads();

    // ---- phase 2: particle updates over the CTA's storage ranges ----
    const uint32_t c1 = min(c0 + (uint32_t)kCellsPerCta, ncells);
    const T tau_t = T(tau);
    const T gt[3] = {T(g0), T(g1), T(g2)};
    {
        const uint32_t a0 = gstart[c0], a1 = gstart[c1];
        for (uint32_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
            V4<T> p = gpos[a];
            if (has_frozen && (gid[a] & kFrozenBit)) {
                gkey[a] = cell_key<T, DIM, EST>(G, p.x, p.y, p.z);
                continue;
            }
            V4<T> v = gvel[a];
            const V4<T> ac = acc[a];
            const uint32_t lc = cell_key<T, DIM, EST>(G, p.x, p.y, p.z) - c0;
            const bool dr = lc < (uint32_t)kCellsPerCta && s_drag[lc];
            T us[3] = {T(0), T(0), T(0)}, ig = T(0);
            if (dr) {
                ig = s_ig[lc];
#pragma unroll
                for (int k = 0; k < DIM; ++k) us[k] = s_us[k][lc];
            }
            gas_particle_update<T, DIM>(G, tau_t, gt, adiabatic, p, v, ac, dr, us, ig);
            gpos[a] = p;
            gvel[a] = v;
            gkey[a] = cell_key<T, DIM, EST>(G, p.x, p.y, p.z);
        }
    }
    {
        const uint32_t j0 = dstart[c0], j1 = dstart[c1];
        for (uint32_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            V4<T> p = dpos[j];
            V4<T> u = dvel[j];
            const uint32_t lc = cell_key<T, DIM, EST>(G, p.x, p.y, p.z) - c0;
            const bool dr = lc < (uint32_t)kCellsPerCta && s_drag[lc];
            T vs[3] = {T(0), T(0), T(0)}, id = T(0);
            if (dr) {
                id = s_id[lc];
#pragma unroll
                for (int k = 0; k < DIM; ++k) vs[k] = s_vs[k][lc];
            }
            dust_particle_update<T, DIM>(G, tau_t, gt, p, u, dr, vs, id);
            dpos[j] = p;
            dvel[j] = u;
            dkey[j] = cell_key<T, DIM, EST>(G, p.x, p.y, p.z);
        }
    }
}

// Reverse mode of the cell drag and the particle update (isothermal gas,
// no viscosity). Inputs, in storage order: lambda of the step's outputs
// x', v' (gas) and x', u' (dust) as V4; outputs: lambda_A (gas, V4),
// lambda_v (gas, written over lgv), lambda_u (dust, over ldu) and
// lambda_t_stop (dust, added to lts). With lv = lambda_v' + tau lambda_x'
// (x' = x + tau v'), for a cell with drag:
//   v_a' = u*' + (v_a + tau (A_a + g) - u*') ig      ig = 1/(1 + rt eps)
//   u_j' = v*' + (u_j + tau g - v*') id              id = 1/(1 + rt)
//   v*' = u*' + w',  u*' = ubar + tau g + rt w',  w' = (vbar - ubar + tau Abar)/den,
//   den = 1 + rt (1 + eps),  rt = tau / t*,  t* = mean (or harmonic mean) of t_j.
template <class T, class A, int DIM>
__global__ void __launch_bounds__(kCellsPerCta)
k_cell_adjoint(Geo<T> G, Phys<T> Ph, A tau, A g0, A g1, A g2, int harmonic, int has_frozen,
               const V4<T> *__restrict__ gvel, const uint32_t *__restrict__ gid, const uint32_t *__restrict__ gstart,
               const V4<T> *__restrict__ acc, const V4<T> *__restrict__ gpos, const V4<T> *__restrict__ dvel,
               const V4<T> *__restrict__ dpos, const uint32_t *__restrict__ dstart, const V4<T> *__restrict__ lgx,
               V4<T> *__restrict__ lgv, const V4<T> *__restrict__ ldx, V4<T> *__restrict__ ldu,
               V4<T> *__restrict__ lA, T *__restrict__ lts)
{
    __shared__ T s_ig[kCellsPerCta], s_id[kCellsPerCta], s_lt[kCellsPerCta], s_tst[kCellsPerCta], s_L[kCellsPerCta];
    __shared__ T s_lv[3][kCellsPerCta], s_lA[3][kCellsPerCta], s_lu[3][kCellsPerCta];
    __shared__ int s_drag[kCellsPerCta];

    const uint32_t ncells = G.ncells;
    const uint32_t c0 = blockIdx.x * kCellsPerCta;
    const uint32_t c = c0 + threadIdx.x;
    const A gv[3] = {g0, g1, g2};
    int drag = 0;
    if (c < ncells) {
        const uint32_t gs = gstart[c], ge = gstart[c + 1];
        const uint32_t ds = dstart[c], de = dstart[c + 1];
        A N = A(0), L = A(0), st = A(0);
        A sv[3] = {A(0), A(0), A(0)}, sa[3] = {A(0), A(0), A(0)}, su[3] = {A(0), A(0), A(0)};
        for (uint32_t a = gs; a < ge; ++a) {
            if (has_frozen && (gid[a] & kFrozenBit)) continue;
            const V4<T> v = gvel[a];
            const V4<T> ac = acc[a];
            N += A(1);
            sv[0] += A(v.x); sa[0] += A(ac.x);
            if (DIM > 1) { sv[1] += A(v.y); sa[1] += A(ac.y); }
            if (DIM > 2) { sv[2] += A(v.z); sa[2] += A(ac.z); }
        }
        for (uint32_t j = ds; j < de; ++j) {
            const V4<T> u = dvel[j];
            L += A(1);
            su[0] += A(u.x);
            if (DIM > 1) su[1] += A(u.y);
            if (DIM > 2) su[2] += A(u.z);
            st += harmonic ? A(1) / A(u.w) : A(u.w);
        }
        drag = (N > A(0) && L > A(0)) ? 1 : 0;
        if (drag) {
            const A eps = A(Ph.m_d) * L / (A(Ph.m_g) * N);
            const A tst = harmonic ? L / st : st / L;
            const A rt = tau / tst;
            const A den = A(1) + rt * (A(1) + eps);
            const A ig = A(1) / (A(1) + rt * eps), id = A(1) / (A(1) + rt);
            A wn[3] = {A(0), A(0), A(0)}, un[3] = {A(0), A(0), A(0)}, vn[3] = {A(0), A(0), A(0)};
            for (int k = 0; k < DIM; ++k) {
                wn[k] = ((sv[k] / N - su[k] / L) + tau * (sa[k] / N)) / den;
                un[k] = su[k] / L + tau * gv[k] + rt * wn[k];
                vn[k] = un[k] + wn[k];
            }
            // sums over the cell's particles of the lambdas reaching u*', v*', ig, id
            A S_un[3] = {A(0), A(0), A(0)}, S_vn[3] = {A(0), A(0), A(0)}, S_ig = A(0), S_id = A(0);
            for (uint32_t a = gs; a < ge; ++a) {
                if (has_frozen && (gid[a] & kFrozenBit)) continue;
                const V4<T> v = gvel[a], ac = acc[a], lx = lgx[a], lv = lgv[a];
                const A l[3] = {A(lv.x) + tau * A(lx.x), A(lv.y) + tau * A(lx.y), A(lv.z) + tau * A(lx.z)};
                const A vv[3] = {A(v.x), A(v.y), A(v.z)}, aa[3] = {A(ac.x), A(ac.y), A(ac.z)};
                for (int k = 0; k < DIM; ++k) {
                    S_un[k] += (A(1) - ig) * l[k];
                    S_ig += (vv[k] + tau * (aa[k] + gv[k]) - un[k]) * l[k];
                }
            }
            for (uint32_t j = ds; j < de; ++j) {
                const V4<T> u = dvel[j], lx = ldx[j], lu = ldu[j];
                const A l[3] = {A(lu.x) + tau * A(lx.x), A(lu.y) + tau * A(lx.y), A(lu.z) + tau * A(lx.z)};
                const A uu[3] = {A(u.x), A(u.y), A(u.z)};
                for (int k = 0; k < DIM; ++k) {
                    S_vn[k] += (A(1) - id) * l[k];
                    S_id += (uu[k] + tau * gv[k] - vn[k]) * l[k];
                }
            }
            A l_rt = A(0), l_den = A(0);
            for (int k = 0; k < DIM; ++k) {
                const A l_vn = S_vn[k];
                const A l_un = S_un[k] + l_vn;
                const A l_wn = l_vn + rt * l_un;
                l_rt += wn[k] * l_un;
                const A l_w = l_wn / den;
                l_den -= wn[k] * l_wn / den;
                s_lv[k][threadIdx.x] = T(l_w / N);                 // lambda of vbar, per gas particle
                s_lA[k][threadIdx.x] = T(tau * l_wn / den / N);    // lambda of Abar, per gas particle
                s_lu[k][threadIdx.x] = T((l_un - l_w) / L);        // lambda of ubar, per dust particle
            }
            l_rt += (A(1) + eps) * l_den;
            l_rt -= eps * ig * ig * S_ig;
            l_rt -= id * id * S_id;
            s_lt[threadIdx.x] = T(-(rt / tst) * l_rt);             // lambda of t*
            s_ig[threadIdx.x] = T(ig);
            s_id[threadIdx.x] = T(id);
            s_tst[threadIdx.x] = T(tst);
            s_L[threadIdx.x] = T(L);
        }
    }
    s_drag[threadIdx.x] = drag;
    __syncthreads();

    const uint32_t c1 = min(c0 + (uint32_t)kCellsPerCta, ncells);
    const T tau_t = T(tau);
    for (uint32_t a = gstart[c0] + threadIdx.x; a < gstart[c1]; a += blockDim.x) {
        V4<T> la;
        la.x = la.y = la.z = la.w = T(0);
        if (has_frozen && (gid[a] & kFrozenBit)) {
            lA[a] = la;
            continue;
        }
        const V4<T> p = gpos[a], lx = lgx[a];
        V4<T> lv = lgv[a];
        lv.x += tau_t * lx.x;
        lv.y += tau_t * lx.y;
        lv.z += tau_t * lx.z;
        const uint32_t lc = cell_key<T, DIM>(G, p.x, p.y, p.z) - c0;
        if (lc < (uint32_t)kCellsPerCta && s_drag[lc]) {
            const T ig = s_ig[lc];
            la.x = tau_t * ig * lv.x + s_lA[0][lc];
            lv.x = ig * lv.x + s_lv[0][lc];
            if (DIM > 1) { la.y = tau_t * ig * lv.y + s_lA[1][lc]; lv.y = ig * lv.y + s_lv[1][lc]; }
            if (DIM > 2) { la.z = tau_t * ig * lv.z + s_lA[2][lc]; lv.z = ig * lv.z + s_lv[2][lc]; }
        } else {
            la.x = tau_t * lv.x;
            la.y = tau_t * lv.y;
            la.z = tau_t * lv.z;
        }
        lv.w = T(0);
        lA[a] = la;
        lgv[a] = lv;
    }
    for (uint32_t j = dstart[c0] + threadIdx.x; j < dstart[c1]; j += blockDim.x) {
        const V4<T> p = dpos[j], lx = ldx[j];
        V4<T> lu = ldu[j];
        lu.x += tau_t * lx.x;
        lu.y += tau_t * lx.y;
        lu.z += tau_t * lx.z;
        const uint32_t lc = cell_key<T, DIM>(G, p.x, p.y, p.z) - c0;
        if (lc < (uint32_t)kCellsPerCta && s_drag[lc]) {
            const T id = s_id[lc];
            lu.x = id * lu.x + s_lu[0][lc];
            if (DIM > 1) lu.y = id * lu.y + s_lu[1][lc];
            if (DIM > 2) lu.z = id * lu.z + s_lu[2][lc];
            // dt*/dt_j: 1/L (arithmetic mean) or t*^2 / (L t_j^2) (harmonic mean)
            const T tj = dvel[j].w;
            const T dtdt = harmonic ? s_tst[lc] * s_tst[lc] / (s_L[lc] * tj * tj) : T(1) / s_L[lc];
            lts[j] += s_lt[lc] * dtdt;
        }
        lu.w = T(0);
        ldu[j] = lu;
    }
}

template <class T, class A, int DIM>
cudaError_t cell_adjoint_t(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G, PhaseBufs &D,
                           const void *acc, const StepArgs &S, const void *lgx, void *lgv, const void *ldx, void *ldu,
                           void *lA, void *lts)
{
    const Geo<T> &Gg = *static_cast<const Geo<T> *>(geo);
    const Phys<T> &Ph = *static_cast<const Phys<T> *>(phys);
    const uint32_t blocks = (Gg.ncells + kCellsPerCta - 1) / kCellsPerCta;
    k_cell_adjoint<T, A, DIM><<<blocks, kCellsPerCta, 0, L.stream>>>(
        Gg, Ph, A(S.tau), A(S.g[0]), A(S.g[1]), A(S.g[2]), S.tstar_mode == TFSPH_TSTAR_HARMONIC, S.has_frozen,
        static_cast<const V4<T> *>(G.vel[G.cur]), G.id[G.cur], G.start, static_cast<const V4<T> *>(acc),
        static_cast<const V4<T> *>(G.pos[G.cur]), static_cast<const V4<T> *>(D.vel[D.cur]),
        static_cast<const V4<T> *>(D.pos[D.cur]), D.start, static_cast<const V4<T> *>(lgx), static_cast<V4<T> *>(lgv),
        static_cast<const V4<T> *>(ldx), static_cast<V4<T> *>(ldu), static_cast<V4<T> *>(lA), static_cast<T *>(lts));
    return cudaGetLastError();
}

template <class T, class A>
cudaError_t cell_adjoint_dim(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G, PhaseBufs &D,
                             const void *acc, const StepArgs &S, const void *lgx, void *lgv, const void *ldx, void *ldu,
                             void *lA, void *lts)
{
    switch (L.dim) {
        case 1: return cell_adjoint_t<T, A, 1>(L, geo, phys, G, D, acc, S, lgx, lgv, ldx, ldu, lA, lts);
        case 2: return cell_adjoint_t<T, A, 2>(L, geo, phys, G, D, acc, S, lgx, lgv, ldx, ldu, lA, lts);
        default: return cell_adjoint_t<T, A, 3>(L, geo, phys, G, D, acc, S, lgx, lgv, ldx, ldu, lA, lts);
    }
}

template <class T, class A, int DIM>
cudaError_t cell_update_t(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G, PhaseBufs &D,
                          const void *acc, const StepArgs &S)
{
    const Geo<T> &Gg = *static_cast<const Geo<T> *>(geo);
    const Phys<T> &Ph = *static_cast<const Phys<T> *>(phys);
    const uint32_t blocks = (Gg.ncells + kCellsPerCta - 1) / kCellsPerCta;
    bool est = true;
    for (int d = 0; d < DIM; ++d) est = est && Gg.est_exact[d];
    auto kern = est ? k_cell_update<T, A, DIM, true> : k_cell_update<T, A, DIM, false>;
    kern<<<blocks, kCellsPerCta, 0, L.stream>>>(
        Gg, Ph, A(S.tau), A(S.g[0]), A(S.g[1]), A(S.g[2]), S.tstar_mode == TFSPH_TSTAR_HARMONIC, S.has_frozen,
        Ph.eos == TFSPH_EOS_ADIABATIC, static_cast<V4<T> *>(G.pos[G.cur]), static_cast<V4<T> *>(G.vel[G.cur]),
        G.id[G.cur], G.key, G.start, static_cast<const V4<T> *>(acc), static_cast<V4<T> *>(D.pos[D.cur]),
        static_cast<V4<T> *>(D.vel[D.cur]), D.key, D.start);
    return cudaGetLastError();
}

template <class T, class A>
cudaError_t cell_update_dim(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G, PhaseBufs &D,
                            const void *acc, const StepArgs &S)
{
    switch (L.dim) {
        case 1: return cell_update_t<T, A, 1>(L, geo, phys, G, D, acc, S);
        case 2: return cell_update_t<T, A, 2>(L, geo, phys, G, D, acc, S);
        default: return cell_update_t<T, A, 3>(L, geo, phys, G, D, acc, S);
    }
}

}  // namespace

cudaError_t launch_cell_adjoint(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G, PhaseBufs &D,
                                const void *acc, const StepArgs &S, const void *lgx, void *lgv, const void *ldx,
                                void *ldu, void *lA, void *lts)
{
    if (L.precision == TFSPH_FP64)
        return cell_adjoint_dim<double, double>(L, geo, phys, G, D, acc, S, lgx, lgv, ldx, ldu, lA, lts);
    if (S.cell_acc == TFSPH_CELL_ACC_FP64)
        return cell_adjoint_dim<float, double>(L, geo, phys, G, D, acc, S, lgx, lgv, ldx, ldu, lA, lts);
    return cell_adjoint_dim<float, float>(L, geo, phys, G, D, acc, S, lgx, lgv, ldx, ldu, lA, lts);
}

cudaError_t launch_cell_update(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G,
                               PhaseBufs &D, const void *acc, const StepArgs &S)
{
    if (L.precision == TFSPH_FP64) return cell_update_dim<double, double>(L, geo, phys, G, D, acc, S);
    if (S.cell_acc == TFSPH_CELL_ACC_FP64) return cell_update_dim<float, double>(L, geo, phys, G, D, acc, S);
    return cell_update_dim<float, float>(L, geo, phys, G, D, acc, S);
}

}  // namespace tfsph
