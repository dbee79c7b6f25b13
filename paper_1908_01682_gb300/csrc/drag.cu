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
#include "tfsph_internal.cuh"

namespace tfsph {
namespace {

template <class T, class A, int DIM>
__global__ void __launch_bounds__(kCellsPerCta)
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
        const uint32_t gs = gstart[c], ge = gstart[c + 1];
        const uint32_t ds = dstart[c], de = dstart[c + 1];
        A N = A(0), L = A(0), st = A(0);
        A sv[3] = {A(0), A(0), A(0)}, sa[3] = {A(0), A(0), A(0)}, su[3] = {A(0), A(0), A(0)};
        for (uint32_t a = gs; a < ge; ++a) {
            if (has_frozen && (gid[a] & kFrozenBit)) continue;
            const V4<T> v = gvel[a];
            const V4<T> ac = acc[a];
            N += A(1);
            sv[0] += A(v.x);
            sa[0] += A(ac.x);
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
            const A invN = A(1) / N, invL = A(1) / L;
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const A vs = sv[k] * invN;
                const A us = su[k] * invL;
                const A ab = sa[k] * invN;
                const A wn = ((vs - us) + tau * ab) / den;
                const A un = us + tau * gv[k] + rt * wn;
                s_us[k][threadIdx.x] = T(un);
                s_vs[k][threadIdx.x] = T(un + wn);
            }
            s_ig[threadIdx.x] = T(A(1) / (A(1) + rt * eps));
            s_id[threadIdx.x] = T(A(1) / (A(1) + rt));
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
                gkey[a] = cell_key<T, DIM>(G, p.x, p.y, p.z);
                continue;
            }
            V4<T> v = gvel[a];
            const V4<T> ac = acc[a];
            const uint32_t lc = cell_key<T, DIM>(G, p.x, p.y, p.z) - c0;
            T vn[3];
            vn[0] = v.x + tau_t * (ac.x + gt[0]);
            vn[1] = DIM > 1 ? v.y + tau_t * (ac.y + gt[1]) : T(0);
            vn[2] = DIM > 2 ? v.z + tau_t * (ac.z + gt[2]) : T(0);
            if (lc < (uint32_t)kCellsPerCta && s_drag[lc]) {
                const T ig = s_ig[lc];
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    const T us = s_us[k][lc];
                    vn[k] = us + (vn[k] - us) * ig;
                }
            }
            v.x = vn[0];
            p.x = p.x + tau_t * vn[0];
            if (G.per[0]) p.x = wrap_periodic(p.x, G.lo[0], G.L[0]);
            if (DIM > 1) {
                v.y = vn[1];
                p.y = p.y + tau_t * vn[1];
                if (G.per[1]) p.y = wrap_periodic(p.y, G.lo[1], G.L[1]);
            }
            if (DIM > 2) {
                v.z = vn[2];
                p.z = p.z + tau_t * vn[2];
                if (G.per[2]) p.z = wrap_periodic(p.z, G.lo[2], G.L[2]);
            }
            if (adiabatic) v.w = v.w + tau_t * ac.w;
            p.w = T(0);
            gpos[a] = p;
            gvel[a] = v;
            gkey[a] = cell_key<T, DIM>(G, p.x, p.y, p.z);
        }
    }
    {
        const uint32_t j0 = dstart[c0], j1 = dstart[c1];
        for (uint32_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            V4<T> p = dpos[j];
            V4<T> u = dvel[j];
            const uint32_t lc = cell_key<T, DIM>(G, p.x, p.y, p.z) - c0;
            T un[3];
            un[0] = u.x + tau_t * gt[0];
            un[1] = DIM > 1 ? u.y + tau_t * gt[1] : T(0);
            un[2] = DIM > 2 ? u.z + tau_t * gt[2] : T(0);
            if (lc < (uint32_t)kCellsPerCta && s_drag[lc]) {
                const T id = s_id[lc];
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    const T vs = s_vs[k][lc];
                    un[k] = vs + (un[k] - vs) * id;
                }
            }
            u.x = un[0];
            p.x = p.x + tau_t * un[0];
            if (G.per[0]) p.x = wrap_periodic(p.x, G.lo[0], G.L[0]);
            if (DIM > 1) {
                u.y = un[1];
                p.y = p.y + tau_t * un[1];
                if (G.per[1]) p.y = wrap_periodic(p.y, G.lo[1], G.L[1]);
            }
            if (DIM > 2) {
                u.z = un[2];
                p.z = p.z + tau_t * un[2];
                if (G.per[2]) p.z = wrap_periodic(p.z, G.lo[2], G.L[2]);
            }
            dpos[j] = p;
            dvel[j] = u;
            dkey[j] = cell_key<T, DIM>(G, p.x, p.y, p.z);
        }
    }
}

template <class T, class A, int DIM>
cudaError_t cell_update_t(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G, PhaseBufs &D,
                          const void *acc, const StepArgs &S)
{
    const Geo<T> &Gg = *static_cast<const Geo<T> *>(geo);
    const Phys<T> &Ph = *static_cast<const Phys<T> *>(phys);
    const uint32_t blocks = (Gg.ncells + kCellsPerCta - 1) / kCellsPerCta;
    k_cell_update<T, A, DIM><<<blocks, kCellsPerCta, 0, L.stream>>>(
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

cudaError_t launch_cell_update(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G,
                               PhaseBufs &D, const void *acc, const StepArgs &S)
{
    if (L.precision == TFSPH_FP64) return cell_update_dim<double, double>(L, geo, phys, G, D, acc, S);
    if (S.cell_acc == TFSPH_CELL_ACC_FP64) return cell_update_dim<float, double>(L, geo, phys, G, D, acc, S);
    return cell_update_dim<float, float>(L, geo, phys, G, D, acc, S);
}

}  // namespace tfsph
