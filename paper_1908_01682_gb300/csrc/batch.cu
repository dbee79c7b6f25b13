// Batched SPH-IDIC step: many independent instances, each with its own box,
// particle counts, h, cell grid, masses, sound speed, tau and g, stepped
// together (the method of Sec. 2.3 applied to every instance at once).
//
// Layout. The instances' particles are concatenated per phase in instance
// order, and their cell grids are concatenated into one key space: the key
// of a particle is the first cell of its instance plus its cell key inside
// the instance. The binning of the single context (count, scan, scatter,
// rank by id) then applies unchanged, and since an instance's cells form
// one contiguous key range, the order by (key, id) keeps each instance's
// particles in one fixed range of storage slots. Work is cut into chunks
// that never straddle an instance: particle chunks for the keys, checks and
// pair sums, cell chunks for the drag. A CTA loads its chunk's instance
// constants into shared memory once.
//
// A step runs in one of two launch forms, both replayed from a captured
// CUDA graph:
//   persistent: one cooperative launch runs all phases, separated by a grid
//     barrier whose waits are bounded by a clock limit: a wait that runs
//     out records TFSPH_E_TIMEOUT and the kernel returns;
//   kernels:    one launch per phase.
// Which half of the double buffer holds the state (the storage parity) is
// kept in device memory, so the same graph serves every step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "drag_ops.cuh"
#include "pair.cuh"
#include "sort_ops.cuh"

using namespace tfsph;

namespace {

constexpr int kItems = 8;              // scan items per thread
constexpr int kMaxBlock = 512;

struct GridBar {
    unsigned int count;
    unsigned int gen;
};

// [begin, end): storage slots (particle chunks) or global cells (cell
// chunks) of instance inst; end - begin <= the CTA size.
struct Chunk {
    uint32_t inst, begin, end, pad;
};

template <class T> struct BInst {
    Geo<T> G;          // geometry of the instance (its own cell grid)
    Phys<T> Ph;
    T hi[3];           // upper box corner, for the input check
    double tau;        // step of the instance
    double g[3];
    uint32_t coff;     // first cell in the batch key space
    uint32_t goff, ng; // gas slots [goff, goff + ng)
    uint32_t doff, nd; // dust slots
    int32_t has_frozen;
    int32_t pad;
};

template <class T> struct BatchArgs {
    const BInst<T> *inst;
    const Chunk *gch, *dch, *cch;  // gas particle, dust particle and cell chunks
    uint32_t ngch, ndch, ncch;
    V4<T> *gpos[2], *gvel[2], *dpos[2], *dvel[2];
    uint32_t *gid[2], *did[2];
    uint32_t *gkey, *dkey, *gcnt, *dcnt, *gstart, *dstart, *gsrc, *dsrc, *gtid, *dtid;
    T *rho;
    V4<T> *acc;
    uint32_t *bsum;
    uint32_t nblk;     // scan tiles per phase (a tile is kItems * CTA size cells)
    uint32_t ncells, ng, nd;
    int *sp;           // storage parity
    int *err;
    GridBar *bar;
    long long spin_limit;  // clock cycles a barrier wait may take
    int harmonic;
};

__device__ __forceinline__ uint32_t thread_rank() { return blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ uint32_t thread_count() { return gridDim.x * blockDim.x; }

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_parity(const int *p) { return *reinterpret_cast<const volatile int *>(p); }

// Grid-wide barrier of a cooperative launch. The last CTA to arrive resets
// the count and advances the generation; the others wait for the generation
// to change, at most spin_limit clock cycles. Returns false (after flagging
// kErrTimeout) when the wait ran out; the caller then returns at once.
template <class T> __device__ bool grid_barrier(const BatchArgs<T> &B)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int g = ld_acquire(&B.bar->gen);
        __threadfence();
        if (atomicAdd(&B.bar->count, 1u) == gridDim.x - 1) {
            atomicExch(&B.bar->count, 0u);
            __threadfence();
            atomicAdd(&B.bar->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (ld_acquire(&B.bar->gen) == g) {
                if (clock64() - t0 > B.spin_limit) {
                    atomicOr(B.err, kErrTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Copies an instance record into shared memory (the whole CTA takes part).
template <class T> __device__ __forceinline__ void load_inst(const BInst<T> *src, BInst<T> &dst)
{
    static_assert(sizeof(BInst<T>) % 4 == 0, "instance record is copied in words");
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(BInst<T>) / 4); k += blockDim.x) d[k] = s[k];
}

// Exclusive scan of one value per thread over a CTA of any multiple of 32
// threads up to 1024; returns the CTA total.
__device__ __forceinline__ uint32_t cta_exclusive_scan(uint32_t v, uint32_t &excl)
{
    __shared__ uint32_t warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = lane < nw ? warp_tot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;
    }
    __syncthreads();
    excl = (wid > 0 ? warp_tot[wid - 1] : 0u) + x - v;
    const uint32_t total = warp_tot[nw - 1];
    __syncthreads();
    return total;
}

// ---------------------------------------------------------------------------
// Phases. Every phase loops over its work with the whole grid, so the same
// body serves a one-launch-per-phase kernel and the persistent kernel.
// ---------------------------------------------------------------------------

// Cell keys in the batch key space (set-up, and after a state load).
template <class T, int DIM> __device__ void ph_keys(const BatchArgs<T> &B, int q, BInst<T> &si)
{
    for (uint32_t c = blockIdx.x; c < B.ngch + B.ndch; c += gridDim.x) {
        const bool gas = c < B.ngch;
        const Chunk ch = gas ? B.gch[c] : B.dch[c - B.ngch];
        __syncthreads();
        load_inst(&B.inst[ch.inst], si);
        __syncthreads();
        const uint32_t i = ch.begin + threadIdx.x;
        if (i < ch.end) {
            const V4<T> p = gas ? B.gpos[q][i] : B.dpos[q][i];
            const uint32_t k = si.coff + cell_key<T, DIM>(si.G, p.x, p.y, p.z);
            if (gas) B.gkey[i] = k;
            else B.dkey[i] = k;
        }
    }
}

// Input check: bit 1 non-finite, bit 2 moving particle outside its box,
// bit 4 t_stop <= 0.
template <class T, int DIM> __device__ void ph_check(const BatchArgs<T> &B, int q, BInst<T> &si, int *flags)
{
    for (uint32_t c = blockIdx.x; c < B.ngch + B.ndch; c += gridDim.x) {
        const bool gas = c < B.ngch;
        const Chunk ch = gas ? B.gch[c] : B.dch[c - B.ngch];
        __syncthreads();
        load_inst(&B.inst[ch.inst], si);
        __syncthreads();
        const uint32_t i = ch.begin + threadIdx.x;
        if (i >= ch.end) continue;
        const V4<T> p = gas ? B.gpos[q][i] : B.dpos[q][i];
        const V4<T> v = gas ? B.gvel[q][i] : B.dvel[q][i];
        const bool frozen = gas && (B.gid[q][i] & kFrozenBit);
        const T xs[3] = {p.x, p.y, p.z}, vs[3] = {v.x, v.y, v.z};
        int f = 0;
        for (int k = 0; k < DIM; ++k) {
            if (!isfinite(xs[k]) || !isfinite(vs[k])) f |= 1;
            else if (!frozen && (xs[k] < si.G.lo[k] || xs[k] >= si.hi[k])) f |= 2;
        }
        if (!isfinite(v.w)) f |= 1;
        if (!gas && !(v.w > T(0))) f |= 4;
        if (f) atomicOr(flags, f);
    }
}

template <class T> __device__ void ph_count(const BatchArgs<T> &B)
{
    for (uint32_t i = thread_rank(); i < B.ng + B.nd; i += thread_count()) {
        const bool gas = i < B.ng;
        const uint32_t k = gas ? B.gkey[i] : B.dkey[i - B.ng];
        if (k < B.ncells) count_add_agg(gas ? &B.gcnt[k] : &B.dcnt[k]);
        else atomicOr(B.err, kErrInternal);
    }
}

template <class T> __device__ void ph_scan_reduce(const BatchArgs<T> &B)
{
    const uint32_t tile = blockDim.x * kItems;
    for (uint32_t t = blockIdx.x; t < 2 * B.nblk; t += gridDim.x) {
        const uint32_t ph = t / B.nblk, b = t - ph * B.nblk;
        const uint32_t *cnt = ph ? B.dcnt : B.gcnt;
        const uint32_t base = b * tile + threadIdx.x * kItems;
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < kItems; ++k)
            if (base + k < B.ncells) s += cnt[base + k];
        uint32_t excl;
        const uint32_t tot = cta_exclusive_scan(s, excl);
        if (threadIdx.x == 0) B.bsum[t] = tot;
    }
}

template <class T> __device__ void ph_scan_top(const BatchArgs<T> &B)
{
    for (uint32_t ph = blockIdx.x; ph < 2; ph += gridDim.x) {
        uint32_t *b = B.bsum + ph * B.nblk;
        uint32_t carry = 0;
        for (uint32_t base = 0; base < B.nblk; base += blockDim.x) {
            const uint32_t i = base + threadIdx.x;
            const uint32_t v = i < B.nblk ? b[i] : 0u;
            uint32_t excl;
            const uint32_t tot = cta_exclusive_scan(v, excl);
            if (i < B.nblk) b[i] = carry + excl;
            carry += tot;
        }
    }
}

template <class T> __device__ void ph_scan_down(const BatchArgs<T> &B)
{
    const uint32_t tile = blockDim.x * kItems;
    for (uint32_t t = blockIdx.x; t < 2 * B.nblk; t += gridDim.x) {
        const uint32_t ph = t / B.nblk, b = t - ph * B.nblk;
        const uint32_t *cnt = ph ? B.dcnt : B.gcnt;
        uint32_t *st = ph ? B.dstart : B.gstart;
        const uint32_t base = b * tile + threadIdx.x * kItems;
        uint32_t v[kItems];
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            v[k] = base + k < B.ncells ? cnt[base + k] : 0u;
            s += v[k];
        }
        uint32_t excl;
        cta_exclusive_scan(s, excl);
        uint32_t run = B.bsum[t] + excl;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            if (base + k < B.ncells) st[base + k] = run;
            run += v[k];
        }
        if (b == 0 && threadIdx.x == 0) st[B.ncells] = ph ? B.nd : B.ng;
    }
}

template <class T> __device__ void ph_scatter(const BatchArgs<T> &B, int q)
{
    for (uint32_t i = thread_rank(); i < B.ng + B.nd; i += thread_count()) {
        if (i < B.ng) scatter_one_agg(i, B.gkey, B.gid[q], B.gcnt, B.gstart, B.gsrc, B.gtid, B.ng, B.err);
        else scatter_one_agg(i - B.ng, B.dkey, B.did[q], B.dcnt, B.dstart, B.dsrc, B.dtid, B.nd, B.err);
    }
}

template <class T> __device__ void ph_gather(const BatchArgs<T> &B, int q)
{
    for (uint32_t s = thread_rank(); s < B.ng + B.nd; s += thread_count()) {
        if (s < B.ng)
            rank_move<T>(s, B.gkey, B.gstart, B.gsrc, B.gtid, B.gpos[q], B.gvel[q], B.gid[q], B.gpos[1 - q],
                         B.gvel[1 - q], B.gid[1 - q], B.ng, B.err);
        else
            rank_move<T>(s - B.ng, B.dkey, B.dstart, B.dsrc, B.dtid, B.dpos[q], B.dvel[q], B.did[q], B.dpos[1 - q],
                         B.dvel[1 - q], B.did[1 - q], B.nd, B.err);
    }
}

// Gas pair sums with storage q: MODE 0 density (and p/rho^2 into pos.w),
// MODE 2/3 pressure (+ viscosity, energy rate) acceleration.
template <class T, int DIM, int MODE> __device__ void ph_pair(const BatchArgs<T> &B, int q, BInst<T> &si)
{
    V4<T> *pos = B.gpos[q];
    const V4<T> *vel = B.gvel[q];
    const uint32_t *id = B.gid[q];
    for (uint32_t c = blockIdx.x; c < B.ngch; c += gridDim.x) {
        const Chunk ch = B.gch[c];
        __syncthreads();
        load_inst(&B.inst[ch.inst], si);
        __syncthreads();
        const uint32_t a = ch.begin + threadIdx.x;
        if (a < ch.end) {
            PairAcc<T, MODE> A;
            const V4<T> pa = pos[a];
            acc_init(A, si.Ph, pa, vel, B.rho, a);
            walk_global<T, DIM, MODE>(A, si.G, si.Ph, pa, pos, vel, B.rho, id, B.gstart + si.coff);
            if (MODE <= 1)
                acc_store<T, MODE>(A, si.Ph, a, si.Ph.m_g, vel, B.rho, reinterpret_cast<T *>(pos), nullptr, nullptr,
                                   nullptr);
            else
                acc_store<T, MODE>(A, si.Ph, a, T(0), vel, nullptr, nullptr, B.acc, nullptr, nullptr);
        }
    }
}

// Tiled gas pair sums of 1D instances (the TFSPH_BATCH_TILED form). The
// particles of a chunk occupy consecutive cells c_first..c_last, so the
// candidates of the whole chunk are the particles of the window of cells
// [c_first - R, c_last + R] (wrapped on a periodic axis): a run of storage,
// plus across the seam one run at the other end of the instance. The window
// is staged in shared memory with a local table of cell starts; each thread
// then walks its particle's candidate cells there, with the arithmetic and
// the neighbour decision of the global walk. A chunk whose window does not
// fit (more than kTileCells cells or cap particles), or an instance whose
// window covers its whole axis, takes the global walk.
constexpr int kTileCells = 1024;

__host__ __device__ constexpr size_t tile_table_bytes() { return ((kTileCells + 1) * 4 + 15) / 16 * 16; }

template <class T, int MODE>
__device__ void ph_pair_tiled(const BatchArgs<T> &B, int q, BInst<T> &si, unsigned char *smem, int cap)
{
    static_assert(MODE == 0 || MODE == 2, "tiled form: density and isothermal force");
    int *lst = reinterpret_cast<int *>(smem);
    V4<T> *sp = reinterpret_cast<V4<T> *>(smem + tile_table_bytes());
    __shared__ int s_win[2];
    V4<T> *pos = B.gpos[q];
    const V4<T> *vel = B.gvel[q];
    const uint32_t *id = B.gid[q];
    for (uint32_t c = blockIdx.x; c < B.ngch; c += gridDim.x) {
        const Chunk ch = B.gch[c];
        __syncthreads();
        load_inst(&B.inst[ch.inst], si);
        __syncthreads();
        const Geo<T> &G = si.G;
        const uint32_t *start = B.gstart + si.coff;
        const int n = G.n[0], R = G.R[0], per = G.per[0];
        if (threadIdx.x == 0) {
            const int c0 = (int)cell_key<T, 1>(G, pos[ch.begin].x, T(0), T(0));
            const int c1 = (int)cell_key<T, 1>(G, pos[ch.end - 1].x, T(0), T(0));
            s_win[0] = c0 - R;
            s_win[1] = c1 - c0 + 2 * R + 1;
        }
        __syncthreads();
        const int w0 = s_win[0], nwc = s_win[1];
        bool tiled = !G.full[0] && nwc <= kTileCells;
        if (tiled) {
            // local cell starts of the window (block-wide scan, kTileCells / CTA rounds at most)
            uint32_t run = 0;
            for (int h0 = 0; h0 < nwc; h0 += blockDim.x) {
                const int h = h0 + (int)threadIdx.x;
                uint32_t cnt = 0;
                if (h < nwc) {
                    int gc = w0 + h;
                    if (per) gc = gc < 0 ? gc + n : (gc >= n ? gc - n : gc);
                    if (gc >= 0 && gc < n) cnt = start[gc + 1] - start[gc];
                }
                uint32_t excl;
                const uint32_t tot = cta_exclusive_scan(cnt, excl);
                if (h < nwc) lst[h] = (int)(run + excl);
                run += tot;
            }
            if (threadIdx.x == 0) lst[nwc] = (int)run;
            tiled = run <= (uint32_t)cap;
            __syncthreads();
            if (tiled) {
                for (int h = threadIdx.x; h < nwc; h += blockDim.x) {
                    int gc = w0 + h;
                    if (per) gc = gc < 0 ? gc + n : (gc >= n ? gc - n : gc);
                    if (gc < 0 || gc >= n) continue;
                    const uint32_t g0 = start[gc];
                    for (int j = lst[h]; j < lst[h + 1]; ++j) sp[j] = pos[g0 + (uint32_t)(j - lst[h])];
                }
                __syncthreads();
            }
        }
        const uint32_t a = ch.begin + threadIdx.x;
        if (a < ch.end) {
            PairAcc<T, MODE> A;
            const V4<T> pa = pos[a];
            acc_init(A, si.Ph, pa, vel, B.rho, a);
            if (tiled) {
                T t;
                const int ca = axis_cell(pa.x, G.lo[0], G.inv_w[0], n, t);
                int olo, ohi;
                x_window(G, t - T(ca), G.lim2, olo, ohi);
                const int hl = max(ca + olo - w0, 0), hh = min(ca + ohi - w0, nwc - 1) + 1;  // window cells [hl, hh)
                // cells h < s0 lie across the low seam, h >= s1 across the high one
                const int s0 = per ? min(max(-w0, 0), nwc) : 0;
                const int s1 = per ? max(min(n - w0, nwc), s0) : nwc;
                auto walk = [&](int h_a, int h_b, auto seam) {
                    for (int j = lst[h_a]; j < lst[h_b]; ++j) {
                        const V4<T> pb = sp[j];
                        T d[3];
                        const T r2 = pair_r2<T, 1, decltype(seam)::value>(G, pa, pb, d);
                        A.add(G, si.Ph, pb, nullptr, T(1), 0u, r2, d);
                    }
                };
                // the global walk's order: wrapped from below, wrapped from above, then the rest,
                // so that both forms sum the same terms in the same order
                if (hl < min(hh, s0)) walk(hl, min(hh, s0), SeamTag<true>{});
                if (max(hl, s1) < hh) walk(max(hl, s1), hh, SeamTag<true>{});
                if (max(hl, s0) < min(hh, s1)) walk(max(hl, s0), min(hh, s1), SeamTag<false>{});
            } else {
                walk_global<T, 1, MODE>(A, si.G, si.Ph, pa, pos, vel, B.rho, id, start);
            }
            if (MODE == 0)
                acc_store<T, MODE>(A, si.Ph, a, si.Ph.m_g, vel, B.rho, reinterpret_cast<T *>(pos), nullptr, nullptr,
                                   nullptr);
            else
                acc_store<T, MODE>(A, si.Ph, a, T(0), vel, nullptr, nullptr, B.acc, nullptr, nullptr);
        }
    }
}

// Cell drag and particle update with storage q (the arithmetic of the
// single context's cell update, per instance); writes the next keys.
template <class T, class A, int DIM>
__device__ void ph_update(const BatchArgs<T> &B, int q, BInst<T> &si, unsigned char *smem)
{
    const int bd = blockDim.x;
    T *s_us = reinterpret_cast<T *>(smem);  // [3][bd]
    T *s_vs = s_us + 3 * bd;                // [3][bd]
    T *s_ig = s_vs + 3 * bd;
    T *s_id = s_ig + bd;
    int *s_drag = reinterpret_cast<int *>(s_id + bd);
    V4<T> *gpos = B.gpos[q], *gvel = B.gvel[q], *dpos = B.dpos[q], *dvel = B.dvel[q];
    const uint32_t *gid = B.gid[q];
    for (uint32_t cc = blockIdx.x; cc < B.ncch; cc += gridDim.x) {
        const Chunk ch = B.cch[cc];
        __syncthreads();
        load_inst(&B.inst[ch.inst], si);
        __syncthreads();
        const A tau = A(si.tau);
        const A gv[3] = {A(si.g[0]), A(si.g[1]), A(si.g[2])};
        const uint32_t cell = ch.begin + threadIdx.x;
        int drag = 0;
        if (cell < ch.end) {
            T un[3] = {T(0), T(0), T(0)}, vn[3] = {T(0), T(0), T(0)}, ig = T(0), id = T(0);
            drag = cell_drag_solve<T, A, DIM>(si.Ph, tau, gv, B.harmonic, si.has_frozen, gvel, gid, B.acc,
                                              B.gstart[cell], B.gstart[cell + 1], dvel, B.dstart[cell],
                                              B.dstart[cell + 1], un, vn, ig, id);
            if (drag) {
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    s_us[k * bd + threadIdx.x] = un[k];
                    s_vs[k * bd + threadIdx.x] = vn[k];
                }
                s_ig[threadIdx.x] = ig;
                s_id[threadIdx.x] = id;
            }
        }
        s_drag[threadIdx.x] = drag;
        __syncthreads();
        const uint32_t c0 = ch.begin - si.coff, ncc = ch.end - ch.begin;
        const T tau_t = T(tau);
        const T gt[3] = {T(gv[0]), T(gv[1]), T(gv[2])};
        const int adiabatic = si.Ph.eos == TFSPH_EOS_ADIABATIC;
        for (uint32_t a = B.gstart[ch.begin] + threadIdx.x; a < B.gstart[ch.end]; a += bd) {
            V4<T> p = gpos[a];
            if (si.has_frozen && (gid[a] & kFrozenBit)) {
                B.gkey[a] = si.coff + cell_key<T, DIM>(si.G, p.x, p.y, p.z);
                continue;
            }
            V4<T> v = gvel[a];
            const V4<T> ac = B.acc[a];
            const uint32_t lc = cell_key<T, DIM>(si.G, p.x, p.y, p.z) - c0;
            const bool dr = lc < ncc && s_drag[lc];
            T us[3] = {T(0), T(0), T(0)}, ig = T(0);
            if (dr) {
                ig = s_ig[lc];
#pragma unroll
                for (int k = 0; k < DIM; ++k) us[k] = s_us[k * bd + lc];
            }
            gas_particle_update<T, DIM>(si.G, tau_t, gt, adiabatic, p, v, ac, dr, us, ig);
            gpos[a] = p;
            gvel[a] = v;
            B.gkey[a] = si.coff + cell_key<T, DIM>(si.G, p.x, p.y, p.z);
        }
        for (uint32_t j = B.dstart[ch.begin] + threadIdx.x; j < B.dstart[ch.end]; j += bd) {
            V4<T> p = dpos[j];
            V4<T> u = dvel[j];
            const uint32_t lc = cell_key<T, DIM>(si.G, p.x, p.y, p.z) - c0;
            const bool dr = lc < ncc && s_drag[lc];
            T vs[3] = {T(0), T(0), T(0)}, id = T(0);
            if (dr) {
                id = s_id[lc];
#pragma unroll
                for (int k = 0; k < DIM; ++k) vs[k] = s_vs[k * bd + lc];
            }
            dust_particle_update<T, DIM>(si.G, tau_t, gt, p, u, dr, vs, id);
            dpos[j] = p;
            dvel[j] = u;
            B.dkey[j] = si.coff + cell_key<T, DIM>(si.G, p.x, p.y, p.z);
        }
    }
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
using Tf = float;

template <int DIM> __global__ void __launch_bounds__(kMaxBlock) k_b_keys(BatchArgs<Tf> B)
{
    __shared__ BInst<Tf> si;
    ph_keys<Tf, DIM>(B, ld_parity(B.sp), si);
}

template <int DIM> __global__ void __launch_bounds__(kMaxBlock) k_b_check(BatchArgs<Tf> B, int *flags)
{
    __shared__ BInst<Tf> si;
    ph_check<Tf, DIM>(B, ld_parity(B.sp), si, flags);
}

__global__ void __launch_bounds__(kMaxBlock) k_b_count(BatchArgs<Tf> B) { ph_count(B); }
__global__ void __launch_bounds__(kMaxBlock) k_b_scan_reduce(BatchArgs<Tf> B) { ph_scan_reduce(B); }
__global__ void __launch_bounds__(kMaxBlock) k_b_scan_top(BatchArgs<Tf> B) { ph_scan_top(B); }
__global__ void __launch_bounds__(kMaxBlock) k_b_scan_down(BatchArgs<Tf> B) { ph_scan_down(B); }
__global__ void __launch_bounds__(kMaxBlock) k_b_scatter(BatchArgs<Tf> B) { ph_scatter(B, ld_parity(B.sp)); }
__global__ void __launch_bounds__(kMaxBlock) k_b_gather(BatchArgs<Tf> B) { ph_gather(B, ld_parity(B.sp)); }

// After the gather the state lives in the other half: the parity flips.
__global__ void k_b_flip(int *sp) { *sp = 1 - *sp; }

template <int DIM, int MODE> __global__ void __launch_bounds__(kMaxBlock) k_b_pair(BatchArgs<Tf> B)
{
    __shared__ BInst<Tf> si;
    ph_pair<Tf, DIM, MODE>(B, ld_parity(B.sp), si);
}

template <int MODE> __global__ void __launch_bounds__(kMaxBlock) k_b_pair_tiled(BatchArgs<Tf> B, int cap)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BInst<Tf> si;
    ph_pair_tiled<Tf, MODE>(B, ld_parity(B.sp), si, smem, cap);
}

template <class A, int DIM> __global__ void __launch_bounds__(kMaxBlock, sizeof(A) == 4 ? 3 : 1) k_b_update(BatchArgs<Tf> B)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BInst<Tf> si;
    ph_update<Tf, A, DIM>(B, ld_parity(B.sp), si, smem);
}

// The whole step in one cooperative launch.
template <class A, int DIM, int FMODE> __global__ void __launch_bounds__(kMaxBlock) k_b_persistent(BatchArgs<Tf> B)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BInst<Tf> si;
    const int q = ld_parity(B.sp);
    ph_count(B);
    if (!grid_barrier(B)) return;
    // every CTA has read the parity: the state moves to the other half below
    if (blockIdx.x == 0 && threadIdx.x == 0) *B.sp = 1 - q;
    ph_scan_reduce(B);
    if (!grid_barrier(B)) return;
    ph_scan_top(B);
    if (!grid_barrier(B)) return;
    ph_scan_down(B);
    if (!grid_barrier(B)) return;
    ph_scatter(B, q);
    if (!grid_barrier(B)) return;
    ph_gather(B, q);
    if (!grid_barrier(B)) return;
    ph_pair<Tf, DIM, 0>(B, 1 - q, si);
    if (!grid_barrier(B)) return;
    ph_pair<Tf, DIM, FMODE>(B, 1 - q, si);
    if (!grid_barrier(B)) return;
    ph_update<Tf, A, DIM>(B, 1 - q, si, smem);
}

template <class A, int DIM, int FMODE> void *persistent_fn() { return (void *)k_b_persistent<A, DIM, FMODE>; }

void *pick_persistent(int dim, bool fp64_cells, bool full)
{
#define TF_P(A, D)                                                                         \
    return full ? persistent_fn<A, D, 3>() : persistent_fn<A, D, 2>();
    if (fp64_cells) {
        if (dim == 1) { TF_P(double, 1) }
        if (dim == 2) { TF_P(double, 2) }
        TF_P(double, 3)
    }
    if (dim == 1) { TF_P(float, 1) }
    if (dim == 2) { TF_P(float, 2) }
    TF_P(float, 3)
#undef TF_P
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct tfsph_batch {
    int dim = 1;
    int n_inst = 0;
    int harmonic = 0;
    bool fp64_cells = false;
    bool full = false;       // some instance needs the viscosity / energy force
    bool adiabatic = false;  // some instance is adiabatic (gas arrays carry e)
    int64_t ng = 0, nd = 0;
    uint32_t ncells = 0;
    std::vector<BInst<Tf>> hinst;
    std::vector<uint32_t> inst_cells;
    PhaseBufs G, D;          // G.cur / D.cur mirror the device parity
    void *rho = nullptr, *acc = nullptr;
    uint32_t *bsum = nullptr;
    BInst<Tf> *dinst = nullptr;
    Chunk *chunks = nullptr;  // gas, dust and cell chunks, sized for the smallest CTA
    size_t chunk_cap = 0;
    uint32_t ngch = 0, ndch = 0, ncch = 0;
    int *d_sp = nullptr, *d_err = nullptr, *d_flags = nullptr;
    GridBar *d_bar = nullptr;
    void *staging = nullptr;
    size_t staging_bytes = 0;
    void *save = nullptr;     // autotuner copy of the state
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int device = 0, sm_count = 1;
    double clock_khz = 2.0e6;
    // launch form
    int mode = TFSPH_BATCH_KERNELS, block = 256, blocks_per_sm = 1, grid = 0;
    long long spin_limit = 0;
    cudaGraphExec_t exec = nullptr;
    bool graph_ok = true;
    bool tau_set = false;
    int64_t steps = 0, launches = 0, device_bytes = 0;
    std::vector<void *> allocs;
    std::string err;
};

namespace {

thread_local std::string g_batch_init_error;

int bfail(tfsph_batch *b, int code, const std::string &msg)
{
    if (b) b->err = msg;
    else g_batch_init_error = msg;
    return code;
}

int bcuda(tfsph_batch *b, cudaError_t e, const char *where)
{
    return bfail(b, e == cudaErrorMemoryAllocation ? TFSPH_E_OOM : TFSPH_E_CUDA,
                 std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define TB_CUDA(b, call)                                    \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return bcuda((b), e_, #call); \
    } while (0)

int balloc(tfsph_batch *b, void **out, size_t bytes)
{
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(out, bytes);
    if (e != cudaSuccess) {
        *out = nullptr;
        return bcuda(b, e, "cudaMalloc");
    }
    b->allocs.push_back(*out);
    b->device_bytes += (int64_t)bytes;
    return TFSPH_OK;
}

LaunchCtx blctx(const tfsph_batch *b, cudaStream_t s)
{
    LaunchCtx L;
    L.stream = s;
    L.precision = TFSPH_FP32;
    L.dim = b->dim;
    L.d_err = b->d_err;
    L.ev = nullptr;
    return L;
}

// Chunk tables for CTAs of `block` threads: runs of at most `block` gas
// slots, dust slots and cells inside one instance.
int build_chunks(tfsph_batch *b, int block)
{
    std::vector<Chunk> gch, dch, cch;
    for (int i = 0; i < b->n_inst; ++i) {
        const BInst<Tf> &I = b->hinst[i];
        for (uint32_t s = 0; s < I.ng; s += block) gch.push_back({(uint32_t)i, I.goff + s, I.goff + std::min(I.ng, s + block), 0});
        for (uint32_t s = 0; s < I.nd; s += block) dch.push_back({(uint32_t)i, I.doff + s, I.doff + std::min(I.nd, s + block), 0});
        const uint32_t nc = b->inst_cells[i];
        for (uint32_t s = 0; s < nc; s += block) cch.push_back({(uint32_t)i, I.coff + s, I.coff + std::min(nc, s + block), 0});
    }
    const size_t total = gch.size() + dch.size() + cch.size();
    if (total > b->chunk_cap) return bfail(b, TFSPH_E_INTERNAL, "chunk table larger than its allocation");
    std::vector<Chunk> all;
    all.reserve(total);
    all.insert(all.end(), gch.begin(), gch.end());
    all.insert(all.end(), dch.begin(), dch.end());
    all.insert(all.end(), cch.begin(), cch.end());
    if (!all.empty())
        TB_CUDA(b, cudaMemcpyAsync(b->chunks, all.data(), all.size() * sizeof(Chunk), cudaMemcpyHostToDevice, b->stream));
    // the host vector dies on return: complete the copy first
    TB_CUDA(b, cudaStreamSynchronize(b->stream));
    b->ngch = (uint32_t)gch.size();
    b->ndch = (uint32_t)dch.size();
    b->ncch = (uint32_t)cch.size();
    return TFSPH_OK;
}

BatchArgs<Tf> args(const tfsph_batch *b)
{
    BatchArgs<Tf> B{};
    B.inst = b->dinst;
    B.gch = b->chunks;
    B.dch = b->chunks + b->ngch;
    B.cch = b->chunks + b->ngch + b->ndch;
    B.ngch = b->ngch;
    B.ndch = b->ndch;
    B.ncch = b->ncch;
    for (int k = 0; k < 2; ++k) {
        B.gpos[k] = static_cast<float4 *>(b->G.pos[k]);
        B.gvel[k] = static_cast<float4 *>(b->G.vel[k]);
        B.dpos[k] = static_cast<float4 *>(b->D.pos[k]);
        B.dvel[k] = static_cast<float4 *>(b->D.vel[k]);
        B.gid[k] = b->G.id[k];
        B.did[k] = b->D.id[k];
    }
    B.gkey = b->G.key;
    B.dkey = b->D.key;
    B.gcnt = b->G.count;
    B.dcnt = b->D.count;
    B.gstart = b->G.start;
    B.dstart = b->D.start;
    B.gsrc = b->G.tmp_src;
    B.dsrc = b->D.tmp_src;
    B.gtid = b->G.tmp_id;
    B.dtid = b->D.tmp_id;
    B.rho = static_cast<float *>(b->rho);
    B.acc = static_cast<float4 *>(b->acc);
    B.bsum = b->bsum;
    B.nblk = (b->ncells + (uint32_t)(b->block * kItems) - 1) / (uint32_t)(b->block * kItems);
    B.ncells = b->ncells;
    B.ng = (uint32_t)b->ng;
    B.nd = (uint32_t)b->nd;
    B.sp = b->d_sp;
    B.err = b->d_err;
    B.bar = b->d_bar;
    B.spin_limit = b->spin_limit;
    B.harmonic = b->harmonic;
    return B;
}

size_t update_smem(int block) { return (size_t)block * (8 * sizeof(float) + sizeof(int)); }

unsigned grid_for_n(int64_t n, int block) { return (unsigned)std::max<int64_t>(1, (n + block - 1) / block); }

template <int DIM> cudaError_t launch_keys_dim(const tfsph_batch *b, const BatchArgs<Tf> &B, cudaStream_t s)
{
    if (B.ngch + B.ndch == 0) return cudaSuccess;
    k_b_keys<DIM><<<B.ngch + B.ndch, b->block, 0, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_batch_keys(const tfsph_batch *b, cudaStream_t s)
{
    const BatchArgs<Tf> B = args(b);
    switch (b->dim) {
        case 1: return launch_keys_dim<1>(b, B, s);
        case 2: return launch_keys_dim<2>(b, B, s);
        default: return launch_keys_dim<3>(b, B, s);
    }
}

cudaError_t launch_batch_check(const tfsph_batch *b, cudaStream_t s, int *flags)
{
    const BatchArgs<Tf> B = args(b);
    if (B.ngch + B.ndch == 0) return cudaSuccess;
    switch (b->dim) {
        case 1: k_b_check<1><<<B.ngch + B.ndch, b->block, 0, s>>>(B, flags); break;
        case 2: k_b_check<2><<<B.ngch + B.ndch, b->block, 0, s>>>(B, flags); break;
        default: k_b_check<3><<<B.ngch + B.ndch, b->block, 0, s>>>(B, flags); break;
    }
    return cudaGetLastError();
}

template <int DIM> cudaError_t launch_pair_dim(const tfsph_batch *b, const BatchArgs<Tf> &B, cudaStream_t s, bool force)
{
    if (B.ngch == 0) return cudaSuccess;
    if (!force) k_b_pair<DIM, 0><<<B.ngch, b->block, 0, s>>>(B);
    else if (b->full) k_b_pair<DIM, 3><<<B.ngch, b->block, 0, s>>>(B);
    else k_b_pair<DIM, 2><<<B.ngch, b->block, 0, s>>>(B);
    return cudaGetLastError();
}

// Staged particles per chunk of the tiled form: the chunk itself, its
// window's halo and room for uneven cells.
int tile_cap(int block) { return 2 * block + 512; }
size_t tile_smem(int block) { return tile_table_bytes() + (size_t)tile_cap(block) * sizeof(float4); }

cudaError_t launch_pair(const tfsph_batch *b, const BatchArgs<Tf> &B, cudaStream_t s, bool force)
{
    if (b->mode == TFSPH_BATCH_TILED && b->dim == 1 && !b->full) {
        if (B.ngch == 0) return cudaSuccess;
        const size_t sm = tile_smem(b->block);
        if (!force) k_b_pair_tiled<0><<<B.ngch, b->block, sm, s>>>(B, tile_cap(b->block));
        else k_b_pair_tiled<2><<<B.ngch, b->block, sm, s>>>(B, tile_cap(b->block));
        return cudaGetLastError();
    }
    switch (b->dim) {
        case 1: return launch_pair_dim<1>(b, B, s, force);
        case 2: return launch_pair_dim<2>(b, B, s, force);
        default: return launch_pair_dim<3>(b, B, s, force);
    }
}

cudaError_t launch_update(const tfsph_batch *b, const BatchArgs<Tf> &B, cudaStream_t s)
{
    if (B.ncch == 0) return cudaSuccess;
    const size_t sm = update_smem(b->block);
    if (b->fp64_cells) {
        switch (b->dim) {
            case 1: k_b_update<double, 1><<<B.ncch, b->block, sm, s>>>(B); break;
            case 2: k_b_update<double, 2><<<B.ncch, b->block, sm, s>>>(B); break;
            default: k_b_update<double, 3><<<B.ncch, b->block, sm, s>>>(B); break;
        }
    } else {
        switch (b->dim) {
            case 1: k_b_update<float, 1><<<B.ncch, b->block, sm, s>>>(B); break;
            case 2: k_b_update<float, 2><<<B.ncch, b->block, sm, s>>>(B); break;
            default: k_b_update<float, 3><<<B.ncch, b->block, sm, s>>>(B); break;
        }
    }
    return cudaGetLastError();
}

// Binning (count, scan, scatter, rank + gather) and the parity flip.
int enqueue_binning(tfsph_batch *b, const BatchArgs<Tf> &B, cudaStream_t s)
{
    const int64_t n = b->ng + b->nd;
    if (n > 0) k_b_count<<<grid_for_n(n, b->block), b->block, 0, s>>>(B);
    k_b_scan_reduce<<<2 * B.nblk, b->block, 0, s>>>(B);
    k_b_scan_top<<<2, b->block, 0, s>>>(B);
    k_b_scan_down<<<2 * B.nblk, b->block, 0, s>>>(B);
    if (n > 0) {
        k_b_scatter<<<grid_for_n(n, b->block), b->block, 0, s>>>(B);
        k_b_gather<<<grid_for_n(n, b->block), b->block, 0, s>>>(B);
    }
    k_b_flip<<<1, 1, 0, s>>>(b->d_sp);
    TB_CUDA(b, cudaGetLastError());
    return TFSPH_OK;
}

// Kernel launches of one step in the current form (what a graph holds).
int64_t launches_per_step(const tfsph_batch *b)
{
    if (b->mode == TFSPH_BATCH_PERSISTENT) return 1;
    const int64_t n = b->ng + b->nd;
    return (n > 0 ? 6 : 3) + 1 + (b->ngch ? 2 : 0) + (b->ncch ? 1 : 0);
}

int enqueue_step(tfsph_batch *b, cudaStream_t s)
{
    const BatchArgs<Tf> B = args(b);
    if (b->mode == TFSPH_BATCH_PERSISTENT) {
        TB_CUDA(b, cudaMemsetAsync(b->d_bar, 0, sizeof(GridBar), s));
        void *fn = pick_persistent(b->dim, b->fp64_cells, b->full);
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)b->grid);
        cfg.blockDim = dim3((unsigned)b->block);
        cfg.dynamicSmemBytes = update_smem(b->block);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        BatchArgs<Tf> a = B;
        void *params[] = {&a};
        TB_CUDA(b, cudaLaunchKernelExC(&cfg, fn, params));
        return TFSPH_OK;
    }
    // kernels: binning (with the flip, so every later phase reads the new parity)
    int rc = enqueue_binning(b, B, s);
    if (rc) return rc;
    TB_CUDA(b, launch_pair(b, B, s, false));
    TB_CUDA(b, launch_pair(b, B, s, true));
    TB_CUDA(b, launch_update(b, B, s));
    return TFSPH_OK;
}

void drop_graph(tfsph_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

// Captures one step into a graph on a private stream; if the capture is
// refused the steps are launched directly.
int capture(tfsph_batch *b)
{
    drop_graph(b);
    b->graph_ok = false;
    if (!b->cap_stream) TB_CUDA(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return TFSPH_OK;
    }
    const int rc = enqueue_step(b, b->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    if (rc || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        b->err.clear();
        return TFSPH_OK;
    }
    const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        b->exec = nullptr;
        cudaGetLastError();
        return TFSPH_OK;
    }
    b->graph_ok = true;
    return TFSPH_OK;
}

int run_steps(tfsph_batch *b, int nsteps)
{
    if (nsteps <= 0) return TFSPH_OK;
    if (!b->exec && b->graph_ok) {
        int rc = capture(b);
        if (rc) return rc;
    }
    for (int k = 0; k < nsteps; ++k) {
        if (b->exec) {
            TB_CUDA(b, cudaGraphLaunch(b->exec, b->stream));
        } else {
            int rc = enqueue_step(b, b->stream);
            if (rc) return rc;
        }
    }
    b->launches += launches_per_step(b) * nsteps;
    b->steps += nsteps;
    if (nsteps & 1) {
        b->G.cur ^= 1;
        b->D.cur ^= 1;
    }
    return TFSPH_OK;
}

// Sets the launch form; the persistent grid is the co-resident CTA count
// (capped by blocks_per_sm per SM).
int configure(tfsph_batch *b, int mode, int block, int blocks_per_sm, double timeout_ms)
{
    if (mode != TFSPH_BATCH_KERNELS && mode != TFSPH_BATCH_PERSISTENT && mode != TFSPH_BATCH_TILED)
        return bfail(b, TFSPH_E_INVALID_ARG, "unknown batch mode");
    if (mode == TFSPH_BATCH_TILED && (b->dim != 1 || b->full))
        return bfail(b, TFSPH_E_INVALID_ARG, "the tiled form takes 1D batches of isothermal gas without viscosity");
    if (block != 128 && block != 256 && block != 512) return bfail(b, TFSPH_E_INVALID_ARG, "block must be 128, 256 or 512");
    if (blocks_per_sm < 1 || blocks_per_sm > 16) return bfail(b, TFSPH_E_INVALID_ARG, "blocks_per_sm must be in [1, 16]");
    if (!(timeout_ms >= 0) || !std::isfinite(timeout_ms)) return bfail(b, TFSPH_E_INVALID_ARG, "timeout must be finite and >= 0");
    drop_graph(b);
    b->graph_ok = true;
    b->mode = mode;
    b->block = block;
    b->blocks_per_sm = blocks_per_sm;
    b->spin_limit = (long long)(timeout_ms * b->clock_khz);
    int rc = build_chunks(b, block);
    if (rc) return rc;
    b->grid = 0;
    if (mode == TFSPH_BATCH_PERSISTENT) {
        int occ = 0;
        TB_CUDA(b, cudaFuncSetAttribute(pick_persistent(b->dim, b->fp64_cells, b->full),
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)update_smem(kMaxBlock)));
        TB_CUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pick_persistent(b->dim, b->fp64_cells, b->full),
                                                                 block, update_smem(block)));
        if (occ < 1) return bfail(b, TFSPH_E_INVALID_ARG, "the persistent kernel does not fit an SM at this block size");
        b->grid = std::min(occ, blocks_per_sm) * b->sm_count;
    }
    if (mode == TFSPH_BATCH_TILED) {
        TB_CUDA(b, cudaFuncSetAttribute(k_b_pair_tiled<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)tile_smem(kMaxBlock)));
        TB_CUDA(b, cudaFuncSetAttribute(k_b_pair_tiled<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)tile_smem(kMaxBlock)));
    }
    return TFSPH_OK;
}

// Snapshot of the state (current half) for the autotuner.
size_t save_bytes(const tfsph_batch *b) { return (size_t)(b->ng + b->nd) * (2 * sizeof(float4) + 8); }

int copy_state(tfsph_batch *b, bool to_save)
{
    char *p = static_cast<char *>(b->save);
    for (PhaseBufs *P : {&b->G, &b->D}) {
        const size_t n = (size_t)P->n;
        void *parts[4] = {P->pos[P->cur], P->vel[P->cur], P->id[P->cur], P->key};
        const size_t sz[4] = {n * sizeof(float4), n * sizeof(float4), n * 4, n * 4};
        for (int k = 0; k < 4; ++k) {
            if (sz[k]) {
                if (to_save) TB_CUDA(b, cudaMemcpyAsync(p, parts[k], sz[k], cudaMemcpyDeviceToDevice, b->stream));
                else TB_CUDA(b, cudaMemcpyAsync(parts[k], p, sz[k], cudaMemcpyDeviceToDevice, b->stream));
            }
            p += sz[k];
        }
    }
    return TFSPH_OK;
}

// Host parity -> device parity (after a restore).
int push_parity(tfsph_batch *b)
{
    static const int parity[2] = {0, 1};
    TB_CUDA(b, cudaMemcpyAsync(b->d_sp, &parity[b->G.cur], sizeof(int), cudaMemcpyHostToDevice, b->stream));
    return TFSPH_OK;
}

}  // namespace

extern "C" {

int tfsph_batch_init(tfsph_batch **out, const tfsph_params *params, const int64_t *n_gas, const int64_t *n_dust,
                     int32_t n_inst, const void *const *gas, const void *const *dust, const uint8_t *frozen,
                     int mem_kind)
{
    if (!out) return bfail(nullptr, TFSPH_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!params || !n_gas || !n_dust || n_inst < 1) return bfail(nullptr, TFSPH_E_INVALID_ARG, "need n_inst >= 1 and the per-instance arrays");
    if (mem_kind != TFSPH_MEM_HOST && mem_kind != TFSPH_MEM_DEVICE) return bfail(nullptr, TFSPH_E_INVALID_ARG, "bad mem_kind");
    const tfsph_params &p0 = params[0];
    int64_t ng = 0, nd = 0;
    uint64_t ncells = 0;
    bool adiabatic = false, full = false;
    for (int i = 0; i < n_inst; ++i) {
        const tfsph_params &p = params[i];
        std::string why;
        int rc = validate_params(&p, n_gas[i], n_dust[i], why);
        if (rc) return bfail(nullptr, rc, "instance " + std::to_string(i) + ": " + why);
        if (p.dim != p0.dim || p.precision != TFSPH_FP32 || p.tstar_mode != p0.tstar_mode || p.cell_acc != p0.cell_acc)
            return bfail(nullptr, TFSPH_E_INVALID_ARG,
                         "every instance of a batch needs the same dim, tstar_mode and cell_acc, and FP32 precision");
        if (p.drag != TFSPH_DRAG_IDIC)
            return bfail(nullptr, TFSPH_E_INVALID_ARG, "batches run the IDIC drag");
        int nc3[3];
        ncells += cell_grid(p, nc3);
        ng += n_gas[i];
        nd += n_dust[i];
        adiabatic = adiabatic || p.eos == TFSPH_EOS_ADIABATIC;
        full = full || p.eos == TFSPH_EOS_ADIABATIC || p.av_alpha > 0 || p.av_beta > 0;
    }
    if (ng >= ((int64_t)1 << 31) || nd >= ((int64_t)1 << 31)) return bfail(nullptr, TFSPH_E_INVALID_ARG, "batch particle counts must stay below 2^31");
    if (ncells > 1000000000ull) return bfail(nullptr, TFSPH_E_INVALID_ARG, "too many cells in the batch (> 1e9)");
    if ((ng > 0 && !gas) || (nd > 0 && !dust)) return bfail(nullptr, TFSPH_E_INVALID_ARG, "NULL array list");

    tfsph_batch *b = new (std::nothrow) tfsph_batch();
    if (!b) return bfail(nullptr, TFSPH_E_OOM, "host allocation failed");
    auto bail = [&](int code) {
        g_batch_init_error = b->err;
        tfsph_batch_destroy(b);
        return code;
    };
    b->dim = p0.dim;
    b->n_inst = n_inst;
    b->harmonic = p0.tstar_mode == TFSPH_TSTAR_HARMONIC;
    b->fp64_cells = p0.cell_acc == TFSPH_CELL_ACC_FP64;
    b->full = full;
    b->adiabatic = adiabatic;
    b->ng = ng;
    b->nd = nd;
    b->ncells = (uint32_t)ncells;
    b->hinst.resize(n_inst);
    b->inst_cells.resize(n_inst);
    uint32_t coff = 0, goff = 0, doff = 0;
    for (int i = 0; i < n_inst; ++i) {
        const tfsph_params &p = params[i];
        BInst<Tf> &I = b->hinst[i];
        memset(&I, 0, sizeof I);
        int nc3[3];
        const uint32_t nc = cell_grid(p, nc3);
        make_geo_phys<Tf>(p, nc3, nc, I.G, I.Ph);
        for (int d = 0; d < 3; ++d) I.hi[d] = d < p.dim ? (Tf)p.hi[d] : Tf(1);
        I.tau = 0.0;
        I.coff = coff;
        I.goff = goff;
        I.ng = (uint32_t)n_gas[i];
        I.doff = doff;
        I.nd = (uint32_t)n_dust[i];
        b->inst_cells[i] = nc;
        coff += nc;
        goff += (uint32_t)n_gas[i];
        doff += (uint32_t)n_dust[i];
    }
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) return bail(bcuda(b, e, "cudaGetDevice"));
    cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    int khz = 0;
    if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, b->device) == cudaSuccess && khz > 0) b->clock_khz = khz;
    b->spin_limit = (long long)(2000.0 * b->clock_khz);  // 2 s

    int rc;
    void *tmp;
    for (PhaseBufs *P : {&b->G, &b->D}) {
        P->n = P == &b->G ? ng : nd;
        const size_t n = (size_t)P->n;
        for (int k = 0; k < 2; ++k) {
            if ((rc = balloc(b, &P->pos[k], n * sizeof(float4)))) return bail(rc);
            if ((rc = balloc(b, &P->vel[k], n * sizeof(float4)))) return bail(rc);
            if ((rc = balloc(b, &tmp, n * 4))) return bail(rc);
            P->id[k] = static_cast<uint32_t *>(tmp);
        }
        if ((rc = balloc(b, &tmp, n * 4))) return bail(rc);
        P->key = static_cast<uint32_t *>(tmp);
        if ((rc = balloc(b, &tmp, n * 4))) return bail(rc);
        P->tmp_src = static_cast<uint32_t *>(tmp);
        if ((rc = balloc(b, &tmp, n * 4))) return bail(rc);
        P->tmp_id = static_cast<uint32_t *>(tmp);
        if ((rc = balloc(b, &tmp, (size_t)ncells * 4))) return bail(rc);
        P->count = static_cast<uint32_t *>(tmp);
        if ((rc = balloc(b, &tmp, ((size_t)ncells + 1) * 4))) return bail(rc);
        P->start = static_cast<uint32_t *>(tmp);
        e = cudaMemset(P->count, 0, (size_t)ncells * 4);
        if (e != cudaSuccess) return bail(bcuda(b, e, "cudaMemset"));
        P->cur = 0;
    }
    if ((rc = balloc(b, &b->rho, (size_t)ng * 4))) return bail(rc);
    if ((rc = balloc(b, &b->acc, (size_t)ng * sizeof(float4)))) return bail(rc);
    // scan partials for the smallest CTA (128 threads: tiles of 1024 cells)
    if ((rc = balloc(b, &tmp, 2 * ((size_t)ncells / (128 * kItems) + 2) * 4))) return bail(rc);
    b->bsum = static_cast<uint32_t *>(tmp);
    if ((rc = balloc(b, &tmp, (size_t)n_inst * sizeof(BInst<Tf>)))) return bail(rc);
    b->dinst = static_cast<BInst<Tf> *>(tmp);
    b->chunk_cap = (size_t)(ng / 128 + nd / 128 + ncells / 128) + 3 * (size_t)n_inst + 3;
    if ((rc = balloc(b, &tmp, b->chunk_cap * sizeof(Chunk)))) return bail(rc);
    b->chunks = static_cast<Chunk *>(tmp);
    if ((rc = balloc(b, &tmp, 256))) return bail(rc);
    b->d_sp = static_cast<int *>(tmp);
    b->d_err = b->d_sp + 16;
    b->d_flags = b->d_sp + 32;
    b->d_bar = reinterpret_cast<GridBar *>(b->d_sp + 48);
    e = cudaMemset(b->d_sp, 0, 256);
    if (e != cudaSuccess) return bail(bcuda(b, e, "cudaMemset"));
    const int64_t nmax = std::max<int64_t>(ng, nd);
    b->staging_bytes = (size_t)(2 * p0.dim + 1) * (size_t)nmax * 4 + (size_t)ng + 256;
    if ((rc = balloc(b, &b->staging, b->staging_bytes))) return bail(rc);
    // exact cell-face thresholds of every instance's axes (cell_key), one table
    {
        size_t total = 0;
        for (int i = 0; i < n_inst; ++i)
            for (int d = 0; d < p0.dim; ++d) total += (size_t)b->hinst[i].G.n[d] + 1;
        std::vector<Tf> h(total);
        std::vector<size_t> off((size_t)n_inst * 3, 0);
        size_t at = 0;
        for (int i = 0; i < n_inst; ++i)
            for (int d = 0; d < p0.dim; ++d) {
                off[(size_t)i * 3 + d] = at;
                face_thresholds<Tf>(params[i].lo[d], params[i].hi[d], b->hinst[i].G.n[d], h.data() + at);
                at += (size_t)b->hinst[i].G.n[d] + 1;
            }
        if ((rc = balloc(b, &tmp, total * sizeof(Tf)))) return bail(rc);
        e = cudaMemcpy(tmp, h.data(), total * sizeof(Tf), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return bail(bcuda(b, e, "cudaMemcpy"));
        for (int i = 0; i < n_inst; ++i)
            for (int d = 0; d < p0.dim; ++d) b->hinst[i].G.thr[d] = static_cast<const Tf *>(tmp) + off[(size_t)i * 3 + d];
    }
    e = cudaMemcpy(b->dinst, b->hinst.data(), (size_t)n_inst * sizeof(BInst<Tf>), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(bcuda(b, e, "cudaMemcpy"));
    if ((rc = configure(b, TFSPH_BATCH_KERNELS, 256, 1, 2000.0))) return bail(rc);

    // inputs: concatenated component arrays, packed like the single context's
    LaunchCtx L = blctx(b, b->stream);
    const int ngas_arr = 2 * b->dim + (adiabatic ? 1 : 0), ndust_arr = 2 * b->dim + 1;
    for (int ph = 0; ph < 2; ++ph) {
        PhaseBufs &P = ph == 0 ? b->G : b->D;
        const int narr = ph == 0 ? ngas_arr : ndust_arr;
        const void *const *arrs = ph == 0 ? gas : dust;
        if (P.n == 0) continue;
        std::vector<const void *> dv(narr);
        const uint8_t *dfz = nullptr;
        for (int k = 0; k < narr; ++k)
            if (!arrs[k]) return bail(bfail(b, TFSPH_E_INVALID_ARG, "NULL input array"));
        if (mem_kind == TFSPH_MEM_DEVICE) {
            for (int k = 0; k < narr; ++k) dv[k] = arrs[k];
            dfz = ph == 0 ? frozen : nullptr;
        } else {
            char *base = static_cast<char *>(b->staging);
            for (int k = 0; k < narr; ++k) {
                char *dst = base + (size_t)k * (size_t)P.n * 4;
                e = cudaMemcpyAsync(dst, arrs[k], (size_t)P.n * 4, cudaMemcpyHostToDevice, b->stream);
                if (e != cudaSuccess) return bail(bcuda(b, e, "cudaMemcpyAsync"));
                dv[k] = dst;
            }
            if (ph == 0 && frozen) {
                char *dst = base + (size_t)narr * (size_t)P.n * 4;
                e = cudaMemcpyAsync(dst, frozen, (size_t)P.n, cudaMemcpyHostToDevice, b->stream);
                if (e != cudaSuccess) return bail(bcuda(b, e, "cudaMemcpyAsync"));
                dfz = reinterpret_cast<const uint8_t *>(dst);
            }
        }
        e = launch_pack(L, P, dv.data(), ph == 0 ? (adiabatic ? 1 : 0) : 1, dfz, ph == 0);
        if (e != cudaSuccess) return bail(bcuda(b, e, "pack"));
        e = cudaStreamSynchronize(b->stream);  // the staging area is reused by the next phase
        if (e != cudaSuccess) return bail(bcuda(b, e, "cudaStreamSynchronize"));
    }
    // frozen flags per instance (host input only; device flags: assumed present)
    for (int i = 0; i < n_inst; ++i) {
        BInst<Tf> &I = b->hinst[i];
        if (!frozen) I.has_frozen = 0;
        else if (mem_kind == TFSPH_MEM_DEVICE) I.has_frozen = 1;
        else {
            I.has_frozen = 0;
            for (uint32_t a = 0; a < I.ng && !I.has_frozen; ++a) I.has_frozen = frozen[I.goff + a] != 0;
        }
    }
    e = cudaMemcpy(b->dinst, b->hinst.data(), (size_t)n_inst * sizeof(BInst<Tf>), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(bcuda(b, e, "cudaMemcpy"));
    e = launch_batch_keys(b, b->stream);
    if (e != cudaSuccess) return bail(bcuda(b, e, "keys"));
    e = launch_batch_check(b, b->stream, b->d_flags);
    if (e != cudaSuccess) return bail(bcuda(b, e, "check"));
    int flags = 0;
    e = cudaMemcpy(&flags, b->d_flags, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bail(bcuda(b, e, "cudaMemcpy"));
    if (flags & 1) return bail(bfail(b, TFSPH_E_NONFINITE, "non-finite position, velocity or energy in the input"));
    if (flags & 4) return bail(bfail(b, TFSPH_E_NONFINITE, "dust t_stop must be finite and > 0"));
    if (flags & 2) return bail(bfail(b, TFSPH_E_OUT_OF_DOMAIN, "a moving particle lies outside its instance's box"));
    *out = b;
    return TFSPH_OK;
}

int tfsph_batch_set_stream(tfsph_batch *b, void *stream)
{
    if (!b) return bfail(nullptr, TFSPH_E_INVALID_ARG, "batch is NULL");
    b->stream = static_cast<cudaStream_t>(stream);
    return TFSPH_OK;
}

int tfsph_batch_step(tfsph_batch *b, const double *tau, const double *g, int32_t nsteps)
{
    if (!b) return bfail(nullptr, TFSPH_E_INVALID_ARG, "batch is NULL");
    if (nsteps < 0) return bfail(b, TFSPH_E_INVALID_ARG, "nsteps must be >= 0");
    if (!tau && !b->tau_set) return bfail(b, TFSPH_E_INVALID_ARG, "the first step needs tau");
    bool changed = false;
    for (int i = 0; i < b->n_inst; ++i) {
        BInst<Tf> &I = b->hinst[i];
        if (tau) {
            if (!std::isfinite(tau[i]) || !(tau[i] > 0)) return bfail(b, TFSPH_E_INVALID_ARG, "tau must be finite and > 0");
            if (I.tau != tau[i]) { I.tau = tau[i]; changed = true; }
        }
        if (g)
            for (int k = 0; k < 3; ++k) {
                const double v = k < b->dim ? g[3 * i + k] : 0.0;
                if (!std::isfinite(v)) return bfail(b, TFSPH_E_NONFINITE, "non-finite gravity");
                if (I.g[k] != v) { I.g[k] = v; changed = true; }
            }
    }
    b->tau_set = true;
    if (changed) {
        TB_CUDA(b, cudaMemcpyAsync(b->dinst, b->hinst.data(), b->hinst.size() * sizeof(BInst<Tf>),
                                   cudaMemcpyHostToDevice, b->stream));
        // the host table is rewritten by the next call that changes it
        TB_CUDA(b, cudaStreamSynchronize(b->stream));
    }
    return run_steps(b, nsteps);
}

int tfsph_batch_config(tfsph_batch *b, int32_t mode, int32_t block, int32_t blocks_per_sm, double barrier_timeout_ms)
{
    if (!b) return bfail(nullptr, TFSPH_E_INVALID_ARG, "batch is NULL");
    return configure(b, mode, block, blocks_per_sm, barrier_timeout_ms);
}

int tfsph_batch_autotune(tfsph_batch *b, int32_t steps, int32_t *mode, int32_t *block, int32_t *blocks_per_sm,
                         float *ms_per_step)
{
    if (!b) return bfail(nullptr, TFSPH_E_INVALID_ARG, "batch is NULL");
    if (steps < 1) return bfail(b, TFSPH_E_INVALID_ARG, "steps must be >= 1");
    if (!b->tau_set) return bfail(b, TFSPH_E_INVALID_ARG, "set tau with tfsph_batch_step first (nsteps may be 0)");
    int rc;
    if (!b->save && (rc = balloc(b, &b->save, save_bytes(b)))) return rc;
    const int cur0 = b->G.cur;
    const int64_t steps0 = b->steps, launches0 = b->launches;
    const double timeout_ms = (double)b->spin_limit / b->clock_khz;
    if ((rc = copy_state(b, true))) return rc;
    struct Cand { int mode, block, bps; };
    std::vector<Cand> cands;
    for (int blk : {128, 256, 512}) cands.push_back({TFSPH_BATCH_KERNELS, blk, 1});
    if (b->dim == 1 && !b->full)
        for (int blk : {128, 256, 512}) cands.push_back({TFSPH_BATCH_TILED, blk, 1});
    for (int blk : {128, 256, 512})
        for (int bps : {1, 2, 4}) cands.push_back({TFSPH_BATCH_PERSISTENT, blk, bps});
    cudaEvent_t e0, e1;
    TB_CUDA(b, cudaEventCreate(&e0));
    TB_CUDA(b, cudaEventCreate(&e1));
    float best = 1e30f;
    Cand pick = {b->mode, b->block, b->blocks_per_sm};
    for (const Cand &cd : cands) {
        if (configure(b, cd.mode, cd.block, cd.bps, timeout_ms) != TFSPH_OK) {
            b->err.clear();
            continue;
        }
        if (cd.mode == TFSPH_BATCH_PERSISTENT && b->grid < cd.bps * b->sm_count) continue;  // same grid as a smaller bps
        b->G.cur = b->D.cur = cur0;
        if ((rc = copy_state(b, false)) || (rc = push_parity(b))) break;
        if ((rc = run_steps(b, 1))) break;  // warm-up (and graph capture)
        TB_CUDA(b, cudaEventRecord(e0, b->stream));
        if ((rc = run_steps(b, steps))) break;
        TB_CUDA(b, cudaEventRecord(e1, b->stream));
        TB_CUDA(b, cudaEventSynchronize(e1));
        int err = 0;
        TB_CUDA(b, cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (err) {
            TB_CUDA(b, cudaMemset(b->d_err, 0, sizeof(int)));
            continue;
        }
        float ms = 0;
        TB_CUDA(b, cudaEventElapsedTime(&ms, e0, e1));
        ms /= (float)steps;
        if (ms < best) {
            best = ms;
            pick = cd;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    // restore the state and keep the fastest form
    b->G.cur = b->D.cur = cur0;
    if ((rc = copy_state(b, false)) || (rc = push_parity(b))) return rc;
    if ((rc = configure(b, pick.mode, pick.block, pick.bps, timeout_ms))) return rc;
    TB_CUDA(b, cudaStreamSynchronize(b->stream));
    b->steps = steps0;
    b->launches = launches0;
    if (mode) *mode = pick.mode;
    if (block) *block = pick.block;
    if (blocks_per_sm) *blocks_per_sm = pick.bps;
    if (ms_per_step) *ms_per_step = best;
    return TFSPH_OK;
}

int tfsph_batch_fields(tfsph_batch *b, int field, void *out, int mem_kind)
{
    if (!b) return bfail(nullptr, TFSPH_E_INVALID_ARG, "batch is NULL");
    if (mem_kind != TFSPH_MEM_HOST && mem_kind != TFSPH_MEM_DEVICE) return bfail(b, TFSPH_E_INVALID_ARG, "bad mem_kind");
    const PhaseBufs *P;
    int what, ncomp;
    const void *aux = nullptr;
    LaunchCtx L = blctx(b, b->stream);
    switch (field) {
        case TFSPH_FIELD_POS_G: P = &b->G; what = 0; ncomp = b->dim; break;
        case TFSPH_FIELD_VEL_G: P = &b->G; what = 1; ncomp = b->dim; break;
        case TFSPH_FIELD_ENERGY_G: P = &b->G; what = 2; ncomp = 1; break;
        case TFSPH_FIELD_POS_D: P = &b->D; what = 0; ncomp = b->dim; break;
        case TFSPH_FIELD_VEL_D: P = &b->D; what = 1; ncomp = b->dim; break;
        case TFSPH_FIELD_TSTOP_D: P = &b->D; what = 2; ncomp = 1; break;
        case TFSPH_FIELD_RHO_G: {
            // bin the current state and sum densities; the next step bins
            // the same order again (keys unchanged)
            const BatchArgs<Tf> B = args(b);
            int rc = enqueue_binning(b, B, b->stream);
            if (rc) return rc;
            b->G.cur ^= 1;
            b->D.cur ^= 1;
            // keys for the new storage order (the next step's count and scatter read them)
            TB_CUDA(b, launch_batch_keys(b, b->stream));
            TB_CUDA(b, launch_pair(b, B, b->stream, false));
            P = &b->G; what = 3; ncomp = 1; aux = b->rho;
            break;
        }
        default: return bfail(b, TFSPH_E_INVALID_ARG, "field not available for a batch");
    }
    if (P->n == 0) return TFSPH_OK;
    if (!out) return bfail(b, TFSPH_E_INVALID_ARG, "out is NULL");
    const size_t bytes = (size_t)ncomp * (size_t)P->n * 4;
    if (mem_kind == TFSPH_MEM_DEVICE) {
        TB_CUDA(b, launch_unpack(L, *P, what, out, TFSPH_ORDER_ORIGINAL, aux));
        return TFSPH_OK;
    }
    if (bytes > b->staging_bytes) return bfail(b, TFSPH_E_INTERNAL, "staging too small");
    TB_CUDA(b, launch_unpack(L, *P, what, b->staging, TFSPH_ORDER_ORIGINAL, aux));
    TB_CUDA(b, cudaMemcpyAsync(out, b->staging, bytes, cudaMemcpyDeviceToHost, b->stream));
    TB_CUDA(b, cudaStreamSynchronize(b->stream));
    return TFSPH_OK;
}

int tfsph_batch_info(const tfsph_batch *b, tfsph_batch_info_t *out)
{
    if (!b || !out) return TFSPH_E_INVALID_ARG;
    out->n_inst = b->n_inst;
    out->dim = b->dim;
    out->n_gas = b->ng;
    out->n_dust = b->nd;
    out->n_cells = b->ncells;
    out->mode = b->mode;
    out->block = b->block;
    out->grid = b->grid;
    out->graph = b->exec ? 1 : 0;
    out->steps = b->steps;
    out->launches = b->launches;
    out->device_bytes = b->device_bytes;
    return TFSPH_OK;
}

int tfsph_batch_sync(tfsph_batch *b)
{
    if (!b) return bfail(nullptr, TFSPH_E_INVALID_ARG, "batch is NULL");
    TB_CUDA(b, cudaStreamSynchronize(b->stream));
    int err = 0;
    TB_CUDA(b, cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        TB_CUDA(b, cudaMemset(b->d_err, 0, sizeof(int)));
        if (err & kErrTimeout) return bfail(b, TFSPH_E_TIMEOUT, "a grid barrier wait ran out; the step did not complete");
        return bfail(b, TFSPH_E_INTERNAL, "device-side consistency check failed");
    }
    return TFSPH_OK;
}

const char *tfsph_batch_last_error(const tfsph_batch *b)
{
    return b ? b->err.c_str() : g_batch_init_error.c_str();
}

void tfsph_batch_destroy(tfsph_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (void *p : b->allocs) cudaFree(p);
    delete b;
}

}  // extern "C"
