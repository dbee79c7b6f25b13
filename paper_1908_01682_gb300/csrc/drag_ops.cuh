// Arithmetic of the implicit drag in cell (Sec. 2.3, Eqs. 17-21) shared by the
// single-context cell update and the batched step: the per-cell sums and
// implicit solve, and the per-particle update of each phase.
#pragma once

#include "tfsph_internal.cuh"

namespace tfsph {

// One cell: N, L, sum v, sum u, sum A, sum t_j (or sum 1/t_j) in storage
// order, with accumulator type A, then
//   eps* = m_d L / (m_g N)                                (Eq. 17)
//   t*   = sum t_j / L   (or L / sum 1/t_j)               (Eq. 18)
//   w    = v_* - u_*                                      (Eq. 21)
//   w'   = (w + tau Abar) / (1 + tau (1 + eps*)/t*)
//   u_*' = u_* + tau g + (tau/t*) w',  v_*' = u_*' + w'
// which is the cell average of the implicit Eqs. 19-20. Returns 1 when the
// cell holds moving gas and dust (drag applies) and then sets un = u_*',
// vn = v_*', ig = 1/(1 + tau eps*/t*) and id = 1/(1 + tau/t*).
template <class T, class A, int DIM>
__device__ __forceinline__ int cell_drag_solve(const Phys<T> &Ph, A tau, const A gv[3], int harmonic, int has_frozen,
                                               const V4<T> *__restrict__ gvel, const uint32_t *__restrict__ gid,
                                               const V4<T> *__restrict__ acc, uint32_t gs, uint32_t ge,
                                               const V4<T> *__restrict__ dvel, uint32_t ds, uint32_t de, T un_out[3],
                                               T vn_out[3], T &ig_out, T &id_out)
{
    A N = A(0), L = A(0), st = A(0);
    A sv[3] = {A(0), A(0), A(0)}, sa[3] = {A(0), A(0), A(0)}, su[3] = {A(0), A(0), A(0)};
    auto add_gas = [&](uint32_t idv, const V4<T> &v, const V4<T> &ac) {
        if (has_frozen && (idv & kFrozenBit)) return;
        N += A(1);
        sv[0] += A(v.x);
        sa[0] += A(ac.x);
        if (DIM > 1) { sv[1] += A(v.y); sa[1] += A(ac.y); }
        if (DIM > 2) { sv[2] += A(v.z); sa[2] += A(ac.z); }
    };
    auto add_dust = [&](const V4<T> &u) {
        L += A(1);
        su[0] += A(u.x);
        if (DIM > 1) su[1] += A(u.y);
        if (DIM > 2) su[2] += A(u.z);
        st += harmonic ? A(1) / A(u.w) : A(u.w);
    };
    // the first gas and dust particles are loaded together (the usual cell
    // holds one or a few of each), the rest in storage order
    V4<T> v0{}, a0{}, u0{};
    uint32_t id0 = 0u;
    if (gs < ge) {
        v0 = gvel[gs];
        a0 = acc[gs];
        if (has_frozen) id0 = gid[gs];
    }
    if (ds < de) u0 = dvel[ds];
    if (gs < ge) add_gas(id0, v0, a0);
    for (uint32_t a = gs + 1; a < ge; ++a) add_gas(has_frozen ? gid[a] : 0u, gvel[a], acc[a]);
    if (ds < de) add_dust(u0);
    for (uint32_t j = ds + 1; j < de; ++j) add_dust(dvel[j]);
    if (!(N > A(0) && L > A(0))) return 0;
    const A eps = A(Ph.m_d) * L / (A(Ph.m_g) * N);
    // 1/N and 1/L from one division (N L is an exact product of counts)
    const A invNL = A(1) / (N * L);
    const A invN = L * invNL, invL = N * invNL;
    // rt = tau / t*, with t* = st / L (mean) or L / st (harmonic mean)
    const A rt = harmonic ? tau * st * invL : tau * L / st;
    const A den = A(1) + rt * (A(1) + eps);
    const A invden = A(1) / den;  // one division for the DIM components
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const A vs = sv[k] * invN;
        const A us = su[k] * invL;
        const A ab = sa[k] * invN;
        const A wn = ((vs - us) + tau * ab) * invden;
        const A un = us + tau * gv[k] + rt * wn;
        un_out[k] = T(un);
        vn_out[k] = T(un + wn);
    }
    // 1/(1 + rt eps) and 1/(1 + rt) from one division
    const A dg = A(1) + rt * eps, dd = A(1) + rt;
    const A invgd = A(1) / (dg * dd);
    ig_out = T(dd * invgd);
    id_out = T(dg * invgd);
    return 1;
}

// Gas particle (Eq. 19 solved for v'): v' = u_*' + (v + tau (A + g) - u_*') ig
// in a drag cell, v + tau (A + g) otherwise; e' = e + tau de/dt (adiabatic);
// x' = x + tau v' with the periodic wrap.
template <class T, int DIM>
__device__ __forceinline__ void gas_particle_update(const Geo<T> &G, T tau_t, const T gt[3], int adiabatic, V4<T> &p,
                                                    V4<T> &v, const V4<T> &ac, bool drag, const T us[3], T ig)
{
    T vn[3];
    vn[0] = v.x + tau_t * (ac.x + gt[0]);
    vn[1] = DIM > 1 ? v.y + tau_t * (ac.y + gt[1]) : T(0);
    vn[2] = DIM > 2 ? v.z + tau_t * (ac.z + gt[2]) : T(0);
    if (drag) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) vn[k] = us[k] + (vn[k] - us[k]) * ig;
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
}

// Dust particle (Eq. 20 solved for u'): u' = v_*' + (u + tau g - v_*') id in a
// drag cell, u + tau g otherwise; x' = x + tau u' with the periodic wrap.
template <class T, int DIM>
__device__ __forceinline__ void dust_particle_update(const Geo<T> &G, T tau_t, const T gt[3], V4<T> &p, V4<T> &u,
                                                     bool drag, const T vs[3], T id)
{
    T un[3];
    un[0] = u.x + tau_t * gt[0];
    un[1] = DIM > 1 ? u.y + tau_t * gt[1] : T(0);
    un[2] = DIM > 2 ? u.z + tau_t * gt[2] : T(0);
    if (drag) {
#pragma unroll
        for (int k = 0; k < DIM; ++k) un[k] = vs[k] + (un[k] - vs[k]) * id;
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
}

}  // namespace tfsph
