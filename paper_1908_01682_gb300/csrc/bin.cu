// Binning of both phases into cells (the decomposition into disjoint volumes
// of Sec. 2.3) and the data movement around it.
//
// Sort by (cell key, particle id), in four passes over both phases at once:
//   1. count   : count[key]++ per particle (atomics; the counts are exact).
//   2. scan    : start = exclusive prefix sum of count (reduce / top / down),
//                start[ncells] = n. These are the cell ranges.
//   3. scatter : slot = start[key] + (atomicSub(count[key]) - 1); the order
//                inside a cell is arbitrary here and count returns to zero.
//   4. rank + gather : the rank of a particle inside its cell is the number
//                of the cell's particles with a smaller id, so the final slot
//                start[key] + rank is unique and deterministic; the particle's
//                state is copied there (double buffer).
// Also: packing of user arrays, field export, t_stop updates, input checks
// and the Courant speed reduction.
#include <algorithm>

#include "sort_ops.cuh"

namespace tfsph {
namespace {

template <class T, int DIM>
__global__ void k_keys(Geo<T> G, const V4<T> *__restrict__ pos, int n, uint32_t *__restrict__ key)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const V4<T> p = pos[i];
    key[i] = cell_key<T, DIM>(G, p.x, p.y, p.z);
}

// AGG: the warp's atomics on one counter are combined (cells holding several
// particles of a phase).
template <bool AGG>
__global__ void k_count(const uint32_t *__restrict__ kg, int ng, uint32_t *__restrict__ cg,
                        const uint32_t *__restrict__ kd, int nd, uint32_t *__restrict__ cd)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ng + nd) return;
    uint32_t *c = i < ng ? &cg[kg[i]] : &cd[kd[i - ng]];
    if (AGG) count_add_agg(c);
    else atomicAdd(c, 1u);
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t &excl)
{
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    const uint32_t before = wid > 0 ? warp_tot[wid - 1] : 0u;
    excl = before + x - v;
    const uint32_t total = warp_tot[kScanThreads / 32 - 1];
    __syncthreads();
    return total;
}

static_assert(kScanItems == 8, "the scan kernels move each thread's counts as two 16-byte words");

// The kScanItems counts of cells [base, base + kScanItems) (0 past ncells),
// as two 16-byte loads when the run is whole (base is a multiple of 8 cells).
__device__ __forceinline__ void load_items(const uint32_t *__restrict__ cnt, uint32_t base, uint32_t ncells,
                                           uint32_t v[kScanItems])
{
    if (base + kScanItems <= ncells) {
        const uint4 *src = reinterpret_cast<const uint4 *>(cnt + base);
        const uint4 a = src[0], b = src[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = base + k < ncells ? cnt[base + k] : 0u;
    }
}

// blockIdx.y selects the phase (0 gas, 1 dust).
__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const uint32_t *__restrict__ cg, const uint32_t *__restrict__ cd, uint32_t ncells,
              uint32_t *__restrict__ bsum, uint32_t nblk)
{
    const uint32_t *cnt = blockIdx.y == 0 ? cg : cd;
    const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    load_items(cnt, base, ncells, v);
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s += v[k];
    uint32_t excl;
    const uint32_t tot = block_exclusive_scan(s, excl);
    if (threadIdx.x == 0) bsum[blockIdx.y * nblk + blockIdx.x] = tot;
}

// One block per phase: exclusive scan of the nblk block totals in place.
__global__ void __launch_bounds__(kScanThreads) k_scan_top(uint32_t *__restrict__ bsum, uint32_t nblk)
{
    uint32_t *b = bsum + blockIdx.x * nblk;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < nblk; base += kScanThreads) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nblk ? b[i] : 0u;
        uint32_t excl;
        const uint32_t tot = block_exclusive_scan(v, excl);
        if (i < nblk) b[i] = carry + excl;
        carry += tot;
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_down(const uint32_t *__restrict__ cg, const uint32_t *__restrict__ cd, uint32_t ncells,
            const uint32_t *__restrict__ bsum, uint32_t nblk, uint32_t *__restrict__ sg,
            uint32_t *__restrict__ sd, uint32_t ng, uint32_t nd)
{
    const uint32_t *cnt = blockIdx.y == 0 ? cg : cd;
    uint32_t *st = blockIdx.y == 0 ? sg : sd;
    const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    load_items(cnt, base, ncells, v);
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s += v[k];
    uint32_t excl;
    block_exclusive_scan(s, excl);
    uint32_t run = bsum[blockIdx.y * nblk + blockIdx.x] + excl;
    uint32_t o[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        o[k] = run;
        run += v[k];
    }
    if (base + kScanItems <= ncells) {
        uint4 *dst = reinterpret_cast<uint4 *>(st + base);
        dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
        dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k)
            if (base + k < ncells) st[base + k] = o[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st[ncells] = blockIdx.y == 0 ? ng : nd;
}

template <bool AGG>
__global__ void k_scatter(const uint32_t *__restrict__ kg, const uint32_t *__restrict__ idg,
                          uint32_t *__restrict__ cg, const uint32_t *__restrict__ sg, uint32_t *__restrict__ srcg,
                          uint32_t *__restrict__ tidg, int ng, const uint32_t *__restrict__ kd,
                          const uint32_t *__restrict__ idd, uint32_t *__restrict__ cd,
                          const uint32_t *__restrict__ sd, uint32_t *__restrict__ srcd,
                          uint32_t *__restrict__ tidd, int nd, int *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (AGG) {
        if (i < ng) scatter_one_agg((uint32_t)i, kg, idg, cg, sg, srcg, tidg, (uint32_t)ng, err);
        else if (i < ng + nd) scatter_one_agg((uint32_t)(i - ng), kd, idd, cd, sd, srcd, tidd, (uint32_t)nd, err);
    } else {
        if (i < ng) scatter_one((uint32_t)i, kg, idg, cg, sg, srcg, tidg, (uint32_t)ng, err);
        else if (i < ng + nd) scatter_one((uint32_t)(i - ng), kd, idd, cd, sd, srcd, tidd, (uint32_t)nd, err);
    }
}

template <class T>
__global__ void k_rank_gather(const uint32_t *__restrict__ kg, const uint32_t *__restrict__ sg,
                              const uint32_t *__restrict__ srcg, const uint32_t *__restrict__ tidg,
                              const V4<T> *__restrict__ pg, const V4<T> *__restrict__ vg,
                              const uint32_t *__restrict__ ig, V4<T> *__restrict__ opg, V4<T> *__restrict__ ovg,
                              uint32_t *__restrict__ oig, int ng, const uint32_t *__restrict__ kd,
                              const uint32_t *__restrict__ sd, const uint32_t *__restrict__ srcd,
                              const uint32_t *__restrict__ tidd, const V4<T> *__restrict__ pd,
                              const V4<T> *__restrict__ vd, const uint32_t *__restrict__ id_,
                              V4<T> *__restrict__ opd, V4<T> *__restrict__ ovd, uint32_t *__restrict__ oid, int nd,
                              int *err)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < ng) rank_move<T>((uint32_t)s, kg, sg, srcg, tidg, pg, vg, ig, opg, ovg, oig, (uint32_t)ng, err);
    else if (s < ng + nd)
        rank_move<T>((uint32_t)(s - ng), kd, sd, srcd, tidd, pd, vd, id_, opd, ovd, oid, (uint32_t)nd, err);
}

// Pack component arrays (x.., v.., [w]) into V4 state; id = index (+ frozen bit).
template <class T, int DIM>
__global__ void k_pack(const T *__restrict__ x0, const T *__restrict__ x1, const T *__restrict__ x2,
                       const T *__restrict__ v0, const T *__restrict__ v1, const T *__restrict__ v2,
                       const T *__restrict__ w, const uint8_t *__restrict__ frozen, int n, V4<T> *__restrict__ pos,
                       V4<T> *__restrict__ vel, uint32_t *__restrict__ id)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    V4<T> p, v;
    p.x = x0[i];
    p.y = DIM > 1 ? x1[i] : T(0);
    p.z = DIM > 2 ? x2[i] : T(0);
    p.w = T(0);
    v.x = v0[i];
    v.y = DIM > 1 ? v1[i] : T(0);
    v.z = DIM > 2 ? v2[i] : T(0);
    v.w = w ? w[i] : T(0);
    pos[i] = p;
    vel[i] = v;
    id[i] = (uint32_t)i | ((frozen && frozen[i]) ? kFrozenBit : 0u);
}

// Input checks: bit 1 non-finite, bit 2 moving particle outside [lo, hi),
// bit 4 t_stop <= 0 (dust only).
template <class T, int DIM>
__global__ void k_check(Geo<T> G, const V4<T> *__restrict__ pos, const V4<T> *__restrict__ vel,
                        const uint32_t *__restrict__ id, int n, int is_gas, T hi0, T hi1, T hi2, int *flags)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const V4<T> p = pos[i], v = vel[i];
    int f = 0;
    const T xs[3] = {p.x, p.y, p.z};
    const T vs[3] = {v.x, v.y, v.z};
    const T his[3] = {hi0, hi1, hi2};
    const bool frozen = is_gas && (id[i] & kFrozenBit);
    for (int k = 0; k < DIM; ++k) {
        if (!isfinite(xs[k]) || !isfinite(vs[k])) f |= 1;
        else if (!frozen && (xs[k] < G.lo[k] || xs[k] >= his[k])) f |= 2;
    }
    if (!isfinite(v.w)) f |= 1;
    if (!is_gas && !(v.w > T(0))) f |= 4;
    if (f) atomicOr(flags, f);
}

// Field export: what = 0 position, 1 velocity, 2 vel.w, 3 scalar array aux.
template <class T>
__global__ void k_unpack(const V4<T> *__restrict__ pos, const V4<T> *__restrict__ vel,
                         const uint32_t *__restrict__ id, const T *__restrict__ aux, int n, int dim, int what,
                         int order, T *__restrict__ out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const size_t o = order == TFSPH_ORDER_ORIGINAL ? (size_t)(id[s] & kIdMask) : (size_t)s;
    if (what == 0 || what == 1) {
        const V4<T> v = what == 0 ? pos[s] : vel[s];
        out[o] = v.x;
        if (dim > 1) out[(size_t)n + o] = v.y;
        if (dim > 2) out[2 * (size_t)n + o] = v.z;
    } else if (what == 2) {
        out[o] = vel[s].w;
    } else {
        out[o] = aux[s];
    }
}

// New stopping times in id order into the resident (storage-order) state.
template <class T>
__global__ void k_set_tstop(V4<T> *__restrict__ vel, const uint32_t *__restrict__ id, const T *__restrict__ ts,
                            int n, int *err)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const T t = ts[id[s] & kIdMask];
    if (!(t > T(0)) || !isfinite(t)) atomicOr(err, kErrBadTstop);
    vel[s].w = t;
}

// Per-block max over moving gas of max(|v|, c).
template <class T, int DIM>
__global__ void __launch_bounds__(256)
k_max_speed(Phys<T> Ph, const V4<T> *__restrict__ vel, const uint32_t *__restrict__ id, int n,
            T *__restrict__ partial)
{
    __shared__ T red[256];
    T m = T(0);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        if (id[s] & kFrozenBit) continue;
        const V4<T> v = vel[s];
        T s2 = v.x * v.x;
        if (DIM > 1) s2 += v.y * v.y;
        if (DIM > 2) s2 += v.z * v.z;
        const T sp = sqrt(s2);
        const T c = Ph.eos == TFSPH_EOS_ADIABATIC ? sqrt(Ph.gamma * Ph.gm1 * v.w) : Ph.cs;
        m = fmax(m, fmax(sp, c));
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

template <class T>
__global__ void __launch_bounds__(256) k_max_final(const T *__restrict__ partial, int nblk, T *__restrict__ out)
{
    __shared__ T red[256];
    T m = T(0);
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) m = fmax(m, partial[i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// Adjoint vectors: component-major id order <-> V4 storage order.
// All adjoint inputs of a step into storage order in one launch (gas x, v;
// dust x, u), and the dust t_stop adjoint scratch cleared.
template <class T>
__global__ void k_lam_gather_all(const uint32_t *__restrict__ gid, int ng, const uint32_t *__restrict__ did, int nd,
                                 int dim, const T *__restrict__ lgx, const T *__restrict__ lgv,
                                 const T *__restrict__ ldx, const T *__restrict__ ldu, V4<T> *__restrict__ gx4,
                                 V4<T> *__restrict__ gv4, V4<T> *__restrict__ dx4, V4<T> *__restrict__ du4,
                                 T *__restrict__ lts)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool gas = t < ng;
    const int s = gas ? t : t - ng;
    const int n = gas ? ng : nd;
    if (!gas && s >= nd) return;
    const size_t i = (gas ? gid[s] : did[s]) & kIdMask;
    const T *la = gas ? lgx : ldx;
    const T *lb = gas ? lgv : ldu;
    V4<T> a, b;
    a.x = la[i];
    b.x = lb[i];
    a.y = dim > 1 ? la[(size_t)n + i] : T(0);
    b.y = dim > 1 ? lb[(size_t)n + i] : T(0);
    a.z = dim > 2 ? la[2 * (size_t)n + i] : T(0);
    b.z = dim > 2 ? lb[2 * (size_t)n + i] : T(0);
    a.w = b.w = T(0);
    if (gas) {
        gx4[s] = a;
        gv4[s] = b;
    } else {
        dx4[s] = a;
        du4[s] = b;
        lts[s] = T(0);
    }
}

// All adjoint outputs of a step back to id order in one launch: gas
// lambda_x = gx4 + out (.xyz), lambda_v = gv4; dust lambda_u = du4 and
// lambda_t_stop += lts.
template <class T>
__global__ void k_lam_scatter_all(const uint32_t *__restrict__ gid, int ng, const uint32_t *__restrict__ did, int nd,
                                  int dim, const V4<T> *__restrict__ gx4, const V4<T> *__restrict__ out,
                                  const V4<T> *__restrict__ gv4, const V4<T> *__restrict__ du4,
                                  const T *__restrict__ lts, T *__restrict__ lgx, T *__restrict__ lgv,
                                  T *__restrict__ ldu, T *__restrict__ lt)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ng) {
        const size_t i = gid[t] & kIdMask;
        V4<T> x = gx4[t];
        const V4<T> o = out[t], v = gv4[t];
        x.x += o.x;
        x.y += o.y;
        x.z += o.z;
        lgx[i] = x.x;
        lgv[i] = v.x;
        if (dim > 1) {
            lgx[(size_t)ng + i] = x.y;
            lgv[(size_t)ng + i] = v.y;
        }
        if (dim > 2) {
            lgx[2 * (size_t)ng + i] = x.z;
            lgv[2 * (size_t)ng + i] = v.z;
        }
    } else if (t < ng + nd) {
        const int s = t - ng;
        const size_t i = did[s] & kIdMask;
        const V4<T> u = du4[s];
        ldu[i] = u.x;
        if (dim > 1) ldu[(size_t)nd + i] = u.y;
        if (dim > 2) ldu[2 * (size_t)nd + i] = u.z;
        lt[i] += lts[s];
    }
}

// lambda_rho = dq/drho lambda_q with q = cs^2 / rho (isothermal): -cs^2/rho^2 lambda_q
template <class T>
__global__ void k_lamq_to_lamrho(const V4<T> *__restrict__ lq, const T *__restrict__ rho, int n, T cs2,
                                 T *__restrict__ lrho)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const T r = rho[s];
    lrho[s] = -cs2 / (r * r) * lq[s].w;
}

inline int grid_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

template <class T>
cudaError_t keys_t(const LaunchCtx &L, const void *geo, const PhaseBufs &P)
{
    if (P.n == 0) return cudaSuccess;
    const Geo<T> &G = *static_cast<const Geo<T> *>(geo);
    auto *pos = static_cast<const V4<T> *>(P.pos[P.cur]);
    const int n = (int)P.n;
    switch (L.dim) {
        case 1: k_keys<T, 1><<<grid_for(n, 256), 256, 0, L.stream>>>(G, pos, n, P.key); break;
        case 2: k_keys<T, 2><<<grid_for(n, 256), 256, 0, L.stream>>>(G, pos, n, P.key); break;
        default: k_keys<T, 3><<<grid_for(n, 256), 256, 0, L.stream>>>(G, pos, n, P.key); break;
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t bin_t(const LaunchCtx &L, const void *geo, PhaseBufs &G, PhaseBufs &D, uint32_t *bsum, int64_t nblk)
{
    const Geo<T> &Gm = *static_cast<const Geo<T> *>(geo);
    const int ng = (int)G.n, nd = (int)D.n;
    const int ntot = ng + nd;
    const uint32_t ncells = Gm.ncells;
    // combined atomics pay when a phase has on average more than one particle per cell
    const bool agg = (double)std::max(ng, nd) >= 1.5 * (double)ncells;
    if (ntot > 0) {
        if (agg) k_count<true><<<grid_for(ntot, 256), 256, 0, L.stream>>>(G.key, ng, G.count, D.key, nd, D.count);
        else k_count<false><<<grid_for(ntot, 256), 256, 0, L.stream>>>(G.key, ng, G.count, D.key, nd, D.count);
    }
    if (L.ev) cudaEventRecord(L.ev[1], L.stream);
    dim3 sg((unsigned)nblk, 2);
    k_scan_reduce<<<sg, kScanThreads, 0, L.stream>>>(G.count, D.count, ncells, bsum, (uint32_t)nblk);
    k_scan_top<<<2, kScanThreads, 0, L.stream>>>(bsum, (uint32_t)nblk);
    k_scan_down<<<sg, kScanThreads, 0, L.stream>>>(G.count, D.count, ncells, bsum, (uint32_t)nblk, G.start,
                                                   D.start, (uint32_t)ng, (uint32_t)nd);
    if (L.ev) cudaEventRecord(L.ev[2], L.stream);
    if (ntot > 0) {
        auto scatter = agg ? k_scatter<true> : k_scatter<false>;
        scatter<<<grid_for(ntot, 256), 256, 0, L.stream>>>(G.key, G.id[G.cur], G.count, G.start, G.tmp_src, G.tmp_id,
                                                           ng, D.key, D.id[D.cur], D.count, D.start, D.tmp_src,
                                                           D.tmp_id, nd, L.d_err);
        if (L.ev) cudaEventRecord(L.ev[3], L.stream);
        const int og = G.cur ^ 1, od = D.cur ^ 1;
        k_rank_gather<T><<<grid_for(ntot, 256), 256, 0, L.stream>>>(
            G.key, G.start, G.tmp_src, G.tmp_id, static_cast<const V4<T> *>(G.pos[G.cur]),
            static_cast<const V4<T> *>(G.vel[G.cur]), G.id[G.cur], static_cast<V4<T> *>(G.pos[og]),
            static_cast<V4<T> *>(G.vel[og]), G.id[og], ng, D.key, D.start, D.tmp_src, D.tmp_id,
            static_cast<const V4<T> *>(D.pos[D.cur]), static_cast<const V4<T> *>(D.vel[D.cur]), D.id[D.cur],
            static_cast<V4<T> *>(D.pos[od]), static_cast<V4<T> *>(D.vel[od]), D.id[od], nd, L.d_err);
        G.cur = og;
        D.cur = od;
    } else if (L.ev) {
        cudaEventRecord(L.ev[3], L.stream);
    }
    if (L.ev) cudaEventRecord(L.ev[4], L.stream);
    return cudaGetLastError();
}

template <class T>
cudaError_t pack_t(const LaunchCtx &L, PhaseBufs &P, const void *const *src, int has_w, const uint8_t *frozen)
{
    if (P.n == 0) return cudaSuccess;
    const int n = (int)P.n;
    const int d = L.dim;
    auto c = [&](int k) { return static_cast<const T *>(src[k]); };
    const T *x0 = c(0), *x1 = d > 1 ? c(1) : nullptr, *x2 = d > 2 ? c(2) : nullptr;
    const T *v0 = c(d), *v1 = d > 1 ? c(d + 1) : nullptr, *v2 = d > 2 ? c(d + 2) : nullptr;
    const T *w = has_w ? c(2 * d) : nullptr;
    auto *pos = static_cast<V4<T> *>(P.pos[P.cur]);
    auto *vel = static_cast<V4<T> *>(P.vel[P.cur]);
    switch (d) {
        case 1: k_pack<T, 1><<<grid_for(n, 256), 256, 0, L.stream>>>(x0, x1, x2, v0, v1, v2, w, frozen, n, pos, vel, P.id[P.cur]); break;
        case 2: k_pack<T, 2><<<grid_for(n, 256), 256, 0, L.stream>>>(x0, x1, x2, v0, v1, v2, w, frozen, n, pos, vel, P.id[P.cur]); break;
        default: k_pack<T, 3><<<grid_for(n, 256), 256, 0, L.stream>>>(x0, x1, x2, v0, v1, v2, w, frozen, n, pos, vel, P.id[P.cur]); break;
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t check_t(const LaunchCtx &L, const void *geo, const PhaseBufs &P, int is_gas, int *flags)
{
    if (P.n == 0) return cudaSuccess;
    const Geo<T> &G = *static_cast<const Geo<T> *>(geo);
    const int n = (int)P.n;
    const T hi0 = G.lo[0] + G.L[0], hi1 = G.lo[1] + G.L[1], hi2 = G.lo[2] + G.L[2];
    auto *pos = static_cast<const V4<T> *>(P.pos[P.cur]);
    auto *vel = static_cast<const V4<T> *>(P.vel[P.cur]);
    switch (L.dim) {
        case 1: k_check<T, 1><<<grid_for(n, 256), 256, 0, L.stream>>>(G, pos, vel, P.id[P.cur], n, is_gas, hi0, hi1, hi2, flags); break;
        case 2: k_check<T, 2><<<grid_for(n, 256), 256, 0, L.stream>>>(G, pos, vel, P.id[P.cur], n, is_gas, hi0, hi1, hi2, flags); break;
        default: k_check<T, 3><<<grid_for(n, 256), 256, 0, L.stream>>>(G, pos, vel, P.id[P.cur], n, is_gas, hi0, hi1, hi2, flags); break;
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t max_speed_t(const LaunchCtx &L, const void *phys, const PhaseBufs &G, void *partials, int nblk,
                        void *result)
{
    const Phys<T> &Ph = *static_cast<const Phys<T> *>(phys);
    const int n = (int)G.n;
    auto *vel = static_cast<const V4<T> *>(G.vel[G.cur]);
    switch (L.dim) {
        case 1: k_max_speed<T, 1><<<nblk, 256, 0, L.stream>>>(Ph, vel, G.id[G.cur], n, static_cast<T *>(partials)); break;
        case 2: k_max_speed<T, 2><<<nblk, 256, 0, L.stream>>>(Ph, vel, G.id[G.cur], n, static_cast<T *>(partials)); break;
        default: k_max_speed<T, 3><<<nblk, 256, 0, L.stream>>>(Ph, vel, G.id[G.cur], n, static_cast<T *>(partials)); break;
    }
    k_max_final<T><<<1, 256, 0, L.stream>>>(static_cast<const T *>(partials), nblk, static_cast<T *>(result));
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_keys(const LaunchCtx &L, const void *geo, const PhaseBufs &P)
{
    return L.precision == TFSPH_FP64 ? keys_t<double>(L, geo, P) : keys_t<float>(L, geo, P);
}

cudaError_t launch_bin(const LaunchCtx &L, const void *geo, PhaseBufs &G, PhaseBufs &D, uint32_t *bsum,
                       int64_t nblk)
{
    return L.precision == TFSPH_FP64 ? bin_t<double>(L, geo, G, D, bsum, nblk)
                                     : bin_t<float>(L, geo, G, D, bsum, nblk);
}

cudaError_t launch_pack(const LaunchCtx &L, PhaseBufs &P, const void *const *src, int ncomp_v,
                        const uint8_t *frozen, bool)
{
    return L.precision == TFSPH_FP64 ? pack_t<double>(L, P, src, ncomp_v, frozen)
                                     : pack_t<float>(L, P, src, ncomp_v, frozen);
}

cudaError_t launch_unpack(const LaunchCtx &L, const PhaseBufs &P, int what, void *out, int order, const void *aux)
{
    if (P.n == 0) return cudaSuccess;
    const int n = (int)P.n;
    if (L.precision == TFSPH_FP64) {
        k_unpack<double><<<grid_for(n, 256), 256, 0, L.stream>>>(
            static_cast<const double4a *>(P.pos[P.cur]), static_cast<const double4a *>(P.vel[P.cur]), P.id[P.cur],
            static_cast<const double *>(aux), n, L.dim, what, order, static_cast<double *>(out));
    } else {
        k_unpack<float><<<grid_for(n, 256), 256, 0, L.stream>>>(
            static_cast<const float4 *>(P.pos[P.cur]), static_cast<const float4 *>(P.vel[P.cur]), P.id[P.cur],
            static_cast<const float *>(aux), n, L.dim, what, order, static_cast<float *>(out));
    }
    return cudaGetLastError();
}

cudaError_t launch_set_tstop(const LaunchCtx &L, PhaseBufs &D, const void *t_stop)
{
    if (D.n == 0) return cudaSuccess;
    const int n = (int)D.n;
    if (L.precision == TFSPH_FP64)
        k_set_tstop<double><<<grid_for(n, 256), 256, 0, L.stream>>>(static_cast<double4a *>(D.vel[D.cur]),
                                                                    D.id[D.cur], static_cast<const double *>(t_stop),
                                                                    n, L.d_err);
    else
        k_set_tstop<float><<<grid_for(n, 256), 256, 0, L.stream>>>(static_cast<float4 *>(D.vel[D.cur]), D.id[D.cur],
                                                                   static_cast<const float *>(t_stop), n, L.d_err);
    return cudaGetLastError();
}

cudaError_t launch_check(const LaunchCtx &L, const void *geo, const PhaseBufs &P, int is_gas, int *flags)
{
    return L.precision == TFSPH_FP64 ? check_t<double>(L, geo, P, is_gas, flags)
                                     : check_t<float>(L, geo, P, is_gas, flags);
}

cudaError_t launch_max_speed(const LaunchCtx &L, const void *phys, const PhaseBufs &G, void *partials, int nblk,
                             void *result)
{
    return L.precision == TFSPH_FP64 ? max_speed_t<double>(L, phys, G, partials, nblk, result)
                                     : max_speed_t<float>(L, phys, G, partials, nblk, result);
}

cudaError_t launch_lam_gather_all(const LaunchCtx &L, const PhaseBufs &G, const PhaseBufs &D, const void *lgx,
                                  const void *lgv, const void *ldx, const void *ldu, void *gx4, void *gv4, void *dx4,
                                  void *du4, void *lts)
{
    const int ng = (int)G.n, nd = (int)D.n;
    if (ng + nd == 0) return cudaSuccess;
    if (L.precision == TFSPH_FP64)
        k_lam_gather_all<double><<<grid_for(ng + nd, 256), 256, 0, L.stream>>>(
            G.id[G.cur], ng, D.id[D.cur], nd, L.dim, static_cast<const double *>(lgx), static_cast<const double *>(lgv),
            static_cast<const double *>(ldx), static_cast<const double *>(ldu), static_cast<double4a *>(gx4),
            static_cast<double4a *>(gv4), static_cast<double4a *>(dx4), static_cast<double4a *>(du4),
            static_cast<double *>(lts));
    else
        k_lam_gather_all<float><<<grid_for(ng + nd, 256), 256, 0, L.stream>>>(
            G.id[G.cur], ng, D.id[D.cur], nd, L.dim, static_cast<const float *>(lgx), static_cast<const float *>(lgv),
            static_cast<const float *>(ldx), static_cast<const float *>(ldu), static_cast<float4 *>(gx4),
            static_cast<float4 *>(gv4), static_cast<float4 *>(dx4), static_cast<float4 *>(du4),
            static_cast<float *>(lts));
    return cudaGetLastError();
}

cudaError_t launch_lam_scatter_all(const LaunchCtx &L, const PhaseBufs &G, const PhaseBufs &D, const void *gx4,
                                   const void *out, const void *gv4, const void *du4, const void *lts, void *lgx,
                                   void *lgv, void *ldu, void *lt)
{
    const int ng = (int)G.n, nd = (int)D.n;
    if (ng + nd == 0) return cudaSuccess;
    if (L.precision == TFSPH_FP64)
        k_lam_scatter_all<double><<<grid_for(ng + nd, 256), 256, 0, L.stream>>>(
            G.id[G.cur], ng, D.id[D.cur], nd, L.dim, static_cast<const double4a *>(gx4),
            static_cast<const double4a *>(out), static_cast<const double4a *>(gv4), static_cast<const double4a *>(du4),
            static_cast<const double *>(lts), static_cast<double *>(lgx), static_cast<double *>(lgv),
            static_cast<double *>(ldu), static_cast<double *>(lt));
    else
        k_lam_scatter_all<float><<<grid_for(ng + nd, 256), 256, 0, L.stream>>>(
            G.id[G.cur], ng, D.id[D.cur], nd, L.dim, static_cast<const float4 *>(gx4), static_cast<const float4 *>(out),
            static_cast<const float4 *>(gv4), static_cast<const float4 *>(du4), static_cast<const float *>(lts),
            static_cast<float *>(lgx), static_cast<float *>(lgv), static_cast<float *>(ldu), static_cast<float *>(lt));
    return cudaGetLastError();
}

cudaError_t launch_lamq_to_lamrho(const LaunchCtx &L, const PhaseBufs &P, const void *lq, const void *rho, double cs2,
                                  void *lrho)
{
    if (P.n == 0) return cudaSuccess;
    const int n = (int)P.n;
    if (L.precision == TFSPH_FP64)
        k_lamq_to_lamrho<double><<<grid_for(n, 256), 256, 0, L.stream>>>(static_cast<const double4a *>(lq),
                                                                         static_cast<const double *>(rho), n, cs2,
                                                                         static_cast<double *>(lrho));
    else
        k_lamq_to_lamrho<float><<<grid_for(n, 256), 256, 0, L.stream>>>(static_cast<const float4 *>(lq),
                                                                        static_cast<const float *>(rho), n, (float)cs2,
                                                                        static_cast<float *>(lrho));
    return cudaGetLastError();
}

cudaError_t launch_debug_keys(const LaunchCtx &L, const void *geo, const PhaseBufs &P, uint32_t *out)
{
    PhaseBufs Q = P;
    Q.key = out;
    return launch_keys(L, geo, Q);
}

}  // namespace tfsph
