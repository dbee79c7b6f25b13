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

#include "pair.cuh"

namespace tfsph {
namespace {

constexpr int kTileThreads = 256;
// Shared memory of a tile that stages positions only (density, isothermal
// force): 4 CTAs per SM, each with its static arrays and the 1 KB the
// hardware reserves, within the SM's 228 KB (4 x (56832 + 64 + 1024) bytes).
constexpr int kTileSmemPos = 56832;

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

// Bytes of the 16-bit halo-cell offsets (nhalo + 1 of them), padded to 4.
__host__ __device__ constexpr long lstart_bytes(long nhalo) { return (2 * (nhalo + 1) + 3) / 4 * 4; }

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
// a[m] receives the total, which is also returned (exact in int when the
// 16-bit form truncates the stored sums).
template <class E>
__device__ int block_scan_smem(E *a, int m, int *wsum)
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
    const int total = wsum[(nth >> 5) - 1];
    int run = (wid > 0 ? wsum[wid - 1] : 0) + x - s;
    for (int i = b0; i < b1; ++i) {
        const int v = a[i];
        a[i] = (E)run;
        run += v;
    }
    if (tid == nth - 1) a[m] = (E)run;
    __syncthreads();
    return total;
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

// Appends the neighbours the density walk finds to the particle's list:
// entry n goes to slot n mod 4 of group n / 4 (16-bit stores; the force pass
// reads whole groups). Groups beyond cap entries go to the tile's spare
// group (never read), which keeps the store unconditional.
struct NbRec {
    unsigned long long *base;  // group 0 of the particle
    uint32_t stride;           // owned_cap ((cap + 1) * owned_cap < 2^31: slot offsets fit 32 bits)
    int gcap;                  // cap / 4: the spare group
    int n;
    __device__ __forceinline__ void push(int j, bool seam)
    {
        const uint32_t g = (uint32_t)min(n >> 2, gcap);
        reinterpret_cast<uint16_t *>(base)[((g * stride) << 2) + (uint32_t)(n & 3)] =
            (uint16_t)((uint32_t)j | (seam ? kNbSeam : 0u));
        ++n;
    }
};

template <class T, int DIM, int MODE, bool SEAM, bool REC>
__device__ __forceinline__ void walk_smem_range(PairAcc<T, MODE> &A, const Geo<T> &G, const Phys<T> &Ph,
                                                const V4<T> &pa, const V4<T> *spos, const V4<T> *svel,
                                                const T *srho, const uint32_t *sid, int j0, int j1, NbRec *rec)
{
    // a row holds a few candidates: no unrolled prologue or remainder
#pragma unroll 1
    for (int j = j0; j < j1; ++j) {
        const V4<T> pb = spos[j];
        T d[3];
        const T r2 = pair_r2<T, DIM, SEAM>(G, pa, pb, d);
        if (REC) {
            if (r2 < G.h2x4) {
                A.add(G, Ph, pb, nullptr, T(1), 0u, r2, d);
                rec->push(j, SEAM);
            }
        } else if (ModeUses<MODE>::vel || ModeUses<MODE>::rho) {
            if (r2 < G.h2x4)
                A.add(G, Ph, pb, ModeUses<MODE>::vel ? &svel[j] : nullptr, ModeUses<MODE>::rho ? srho[j] : T(1), 0u,
                      r2, d);
        } else {
            A.add(G, Ph, pb, nullptr, T(1), MODE == 1 ? sid[j] : 0u, r2, d);
        }
    }
}

// Candidate walk of one owned particle over the staged tile (REC: the
// density pass recording the neighbour list; SEAMLESS: no halo cell of the
// tile lies across a periodic seam, or the tile was staged with its seam
// shifts, so every row is one plain range). Each row is walked in the order
// of its staged cells in either case.
template <class T, int DIM, int MODE, bool REC, bool SEAMLESS>
__device__ __forceinline__ void walk_tile(PairAcc<T, MODE> &A, const Geo<T> &G, const Phys<T> &Ph, const TileCfg &C,
                                          const int c0[3], const V4<T> &pa, const V4<T> &pc, const uint16_t *lstart,
                                          const V4<T> *spos, const V4<T> *svel, const T *srho, const uint32_t *sid,
                                          NbRec *rec)
{
    // pa: the staged (possibly shifted) position the displacements use;
    // pc: the same position in box coordinates, for its cell and window
    T tx_, ty_ = T(0), tz_ = T(0);
    const int cx = axis_cell(pc.x, G.lo[0], G.inv_w[0], G.n[0], tx_);
    const int cy = DIM > 1 ? axis_cell(pc.y, G.lo[1], G.inv_w[1], G.n[1], ty_) : 0;
    const int cz = DIM > 2 ? axis_cell(pc.z, G.lo[2], G.inv_w[2], G.n[2], tz_) : 0;
    const T fx = tx_ - T(cx);
    const T fy = DIM > 1 ? ty_ - T(cy) : T(0);
    const T fz = DIM > 2 ? tz_ - T(cz) : T(0);
    const int hx = cx - c0[0] + G.R[0];
    const int hy = DIM > 1 ? cy - c0[1] + G.R[1] : 0;
    const int hz = DIM > 2 ? cz - c0[2] + G.R[2] : 0;
    // x seam bounds in halo coordinates: cells below sx0 or from sx1 on lie across
    const int sx0 = G.per[0] ? G.R[0] - c0[0] : -1;
    const int sx1 = G.per[0] ? G.n[0] - c0[0] + G.R[0] : C.H[0] + 1;
    // z and y offsets limited by the closed form of the x window; a row may
    // come out one cell wider than an exact slab test, which only adds
    // candidates (each pair is decided by its own r^2 < 4h^2)
    int oz0 = 0, oz1 = 0;
    if (DIM > 2) {
        const T tz = approx_sqrt(G.lim2) * G.inv_w[2];
        oz1 = min(G.R[2], max(0, floor_int(fz + tz)));
        oz0 = -min(G.R[2], max(0, floor_int(tz - fz + T(1))));
    }
#pragma unroll 1
    for (int oz = oz0; oz <= oz1; ++oz) {
        T dz2 = T(0);
        int seam_z = 0;
        if (DIM > 2) {
            const T s = slab_dist(oz, fz) * G.w[2];
            dz2 = s * s;
            if (!SEAMLESS) seam_z = halo_seam(G, 2, c0[2], hz + oz);
        }
        int oy0 = 0, oy1 = 0;
        if (DIM > 1) {
            const T ty = approx_sqrt(fmax(G.lim2 - dz2, T(0))) * G.inv_w[1];
            oy1 = min(G.R[1], max(0, floor_int(fy + ty)));
            oy0 = -min(G.R[1], max(0, floor_int(ty - fy + T(1))));
        }
#pragma unroll 1
        for (int oy = oy0; oy <= oy1; ++oy) {
            T dy2 = T(0);
            int seam_y = 0;
            if (DIM > 1) {
                const T s = slab_dist(oy, fy) * G.w[1];
                dy2 = s * s;
                if (!SEAMLESS) seam_y = halo_seam(G, 1, c0[1], hy + oy);
            }
            // x window: the cells whose slab lies within t = sqrt(rem)/w of the
            // particle, (o - fx) <= t for o > 0 and (fx + |o| - 1) <= t for o < 0
            const T t = approx_sqrt(fmax(G.lim2 - dz2 - dy2, T(0))) * G.inv_w[0];
            const int ohi = min(G.R[0], max(0, floor_int(fx + t)));
            const int olo = -min(G.R[0], max(0, floor_int(t - fx + T(1))));
            const int hrow = C.H[0] * ((hy + oy) + C.H[1] * (hz + oz));
            const int u0 = hx + olo, u1 = hx + ohi + 1;  // halo x cells [u0, u1)
            if (SEAMLESS) {
                walk_smem_range<T, DIM, MODE, false, REC>(A, G, Ph, pa, spos, svel, srho, sid, lstart[hrow + u0],
                                                          lstart[hrow + u1], rec);
                continue;
            }
            // [u0, a0) across the low seam, [a0, a1) inside, [a1, u1) across the
            // high seam, in that order (the order of the staged cells, as in the
            // tiles staged with their seam shifts); a row across a y or z seam
            // takes the two-sum displacement over its whole range
            const int a0 = min(max(u0, sx0), u1);
            const int a1 = max(min(u1, sx1), a0);
            if (seam_y | seam_z) {
                walk_smem_range<T, DIM, MODE, true, REC>(A, G, Ph, pa, spos, svel, srho, sid, lstart[hrow + u0],
                                                         lstart[hrow + u1], rec);
                continue;
            }
            if (a0 > u0)
                walk_smem_range<T, DIM, MODE, true, REC>(A, G, Ph, pa, spos, svel, srho, sid, lstart[hrow + u0],
                                                         lstart[hrow + a0], rec);
            if (a1 > a0)
                walk_smem_range<T, DIM, MODE, false, REC>(A, G, Ph, pa, spos, svel, srho, sid, lstart[hrow + a0],
                                                          lstart[hrow + a1], rec);
            if (u1 > a1)
                walk_smem_range<T, DIM, MODE, true, REC>(A, G, Ph, pa, spos, svel, srho, sid, lstart[hrow + a1],
                                                         lstart[hrow + u1], rec);
        }
    }
}

// One particle's sums by the global-memory walk, for tiles whose halo does
// not fit shared memory. Kept out of line so that the rare path does not
// weigh on the register allocation of the tiled walks.
template <class T, int DIM, int MODE>
__device__ __noinline__ void particle_global(const Geo<T> G, const Phys<T> Ph, uint32_t a,
                                             const V4<T> *__restrict__ pos, const V4<T> *__restrict__ vel,
                                             const T *__restrict__ rho, const uint32_t *__restrict__ id,
                                             const uint32_t *__restrict__ start, T mass, T *__restrict__ out_rho,
                                             T *pr_out, V4<T> *__restrict__ out_acc, int32_t *__restrict__ cnt,
                                             uint64_t *__restrict__ fpr)
{
    PairAcc<T, MODE> A;
    const V4<T> pa = pos[a];
    acc_init(A, Ph, pa, vel, rho, a);
    walk_global<T, DIM, MODE>(A, G, Ph, pa, pos, vel, rho, id, start);
    acc_store(A, Ph, a, mass, vel, out_rho, pr_out, out_acc, cnt, fpr);
}

// One particle's sums by the tile walk without recording, for the listing
// passes (density MODE 0, isothermal force MODE 2) when the list does not
// cover the particle; out of line for the same reason as particle_global.
// (The density pass calls it; the force pass keeps its walk inline, where
// the call's register saves cost more than they free.)
template <class T, int DIM, int MODE, bool SEAMLESS>
__device__ __noinline__ void particle_tile(const Geo<T> G, const Phys<T> Ph, const TileCfg C, int c0x, int c0y,
                                           int c0z, const V4<T> pa, const V4<T> pc, uint32_t a, const uint16_t *lstart,
                                           const V4<T> *spos, const V4<T> *__restrict__ vel, T mass,
                                           T *__restrict__ out_rho, T *pr_out, V4<T> *__restrict__ out_acc)
{
    static_assert(MODE == 0 || MODE == 2, "listing passes only");
    PairAcc<T, MODE> A;
    acc_init(A, Ph, pa, vel, static_cast<const T *>(nullptr), a);
    const int c0[3] = {c0x, c0y, c0z};
    walk_tile<T, DIM, MODE, false, SEAMLESS>(A, G, Ph, C, c0, pa, pc, lstart, spos, nullptr, nullptr, nullptr, nullptr);
    acc_store(A, Ph, a, mass, vel, out_rho, pr_out, out_acc, nullptr, nullptr);
}

// Pair sums over a particle's recorded list (groups `e[g * st]` of four
// 16-bit entries, n entries), in the recorded order (SEAMLESS: the tile
// recorded no seam flags).
template <class T, int DIM, int MODE, bool SEAMLESS>
__device__ __forceinline__ void read_list(PairAcc<T, MODE> &A, const Geo<T> &G, const Phys<T> &Ph, const V4<T> &pa,
                                          const V4<T> *spos, const unsigned long long *e, size_t st, int n)
{
    auto pair = [&](uint32_t cur) {
        const V4<T> pb = spos[cur & 0x7FFFu];
        T d[3];
        const T r2 = (!SEAMLESS && (cur & kNbSeam)) ? pair_r2<T, DIM, true>(G, pa, pb, d)
                                                    : pair_r2<T, DIM, false>(G, pa, pb, d);
        A.template add<true>(G, Ph, pb, nullptr, T(1), 0u, r2, d);
    };
    auto quad = [&](unsigned long long w) {
        const uint32_t l = (uint32_t)w, h = (uint32_t)(w >> 32);
        pair(l & 0xFFFFu);
        pair(l >> 16);
        pair(h & 0xFFFFu);
        pair(h >> 16);
    };
    // full groups two at a time through the read-only path, the next two
    // loaded while the current ones are used; then the partial group
    const int ng = n >> 2;
    int g = 0;
    unsigned long long c0, c1, n0 = 0, n1 = 0;
    if (ng >= 2) {
        n0 = __ldg(&e[0]);
        n1 = __ldg(&e[st]);
    }
    for (; g + 2 <= ng; g += 2) {
        c0 = n0;
        c1 = n1;
        if (g + 4 <= ng) {
            n0 = __ldg(&e[(size_t)(g + 2) * st]);
            n1 = __ldg(&e[(size_t)(g + 3) * st]);
        }
        quad(c0);
        quad(c1);
    }
    if (g < ng) quad(__ldg(&e[(size_t)g++ * st]));
    const int m = n & 3;
    if (m) {
        const unsigned long long w = __ldg(&e[(size_t)g * st]);
        for (int u = 0; u < m; ++u) pair((uint32_t)(w >> (16 * u)) & 0xFFFFu);
    }
}

template <class T, int DIM, int MODE>
__global__ void __launch_bounds__(kTileThreads, sizeof(T) == 4 ? ((MODE == 0 || MODE == 2) ? 4 : 3) : 1)
k_pair_tile(Geo<T> G, Phys<T> Ph, TileCfg C, const V4<T> *__restrict__ pos, const V4<T> *__restrict__ vel,
            const T *__restrict__ rho, const uint32_t *__restrict__ id, const uint32_t *__restrict__ start, T mass,
            T *__restrict__ out_rho, T *pr_out, V4<T> *__restrict__ out_acc, int32_t *__restrict__ cnt,
            uint64_t *__restrict__ fpr, NbList nbl)
{
    extern __shared__ __align__(64) unsigned char smem[];
    __shared__ int wsum[kTileThreads / 32];
    // staged offset of every halo cell (16 bits: a staged tile holds at most
    // cap <= 0x7FFF particles), then 32-bit tables
    uint16_t *lstart = reinterpret_cast<uint16_t *>(smem);                     // nhalo + 1
    int *rowpref = reinterpret_cast<int *>(smem + lstart_bytes(C.nhalo));      // nrows + 1
    int *rowg = rowpref + C.nrows + 1;                 // nrows
    const int nhr = C.H[1] * C.H[2];                   // halo rows (along x)
    int *hr_first = rowg + C.nrows;                    // nhr: global start of a halo row
    int *hr_base = hr_first + nhr;                     // nhr + 1: its staged offset
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

    // Periodic seams. A tile whose halo crosses the low seam of axis k stages
    // its wrapped cells at x - L; one whose halo crosses the high seam stages
    // its own cells at x - L and its wrapped ones at x. With lo = 0 every such
    // subtraction is exact (Sterbenz: the coordinates lie within a factor of
    // two of L, for a high seam because the halo lies in the upper half of
    // the box), so each pair's displacement is the plain difference of staged
    // coordinates, the correctly rounded periodic displacement, and the walks
    // take the plain path. Tiles that do not meet this (lo != 0, a halo over
    // both seams) keep the per-pair seam path.
    bool seamless = true, shifted = false;
    int lowk[3] = {0, 0, 0}, highk[3] = {0, 0, 0};
    T orig[3] = {T(0), T(0), T(0)};  // what the owned particles' staged coordinates lack
    {
        bool crosses = false, ok = true;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            if (!G.per[k]) continue;
            lowk[k] = c0[k] < G.R[k];
            highk[k] = c0[k] + ext[k] + G.R[k] > G.n[k];
            if (lowk[k] || highk[k]) {
                crosses = true;
                if (!(G.lo[k] == T(0)) || (lowk[k] && highk[k]) || (highk[k] && 2 * (c0[k] - G.R[k]) < G.n[k]))
                    ok = false;
            }
        }
        if (crosses) {
            if (ok) {
                shifted = true;
#pragma unroll
                for (int k = 0; k < DIM; ++k) orig[k] = highk[k] ? G.L[k] : T(0);
            } else {
                seamless = false;
            }
        }
    }

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
    // a tile whose halo lies inside the grid on every axis (no wrap, no
    // cell outside): each halo row of cells is one contiguous range of the
    // sorted particles, so the rows are counted and copied whole (not for
    // the full force, whose walk then spills a register; and only where the
    // particle area can hold the halo cells' 32-bit starts meanwhile)
    bool interior = MODE != 3 && C.nhalo * 4 <= C.cap * (int)sizeof(V4<T>);
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (c0[k] < G.R[k] || c0[k] + ext[k] + G.R[k] > G.n[k]) interior = false;
    int total;
    if (interior) {
        // the particle area serves as scratch for the global starts until the copy
        int *raw = reinterpret_cast<int *>(smem + C.offset);
        const int gx0 = c0[0] - G.R[0], gy0 = c0[1] - G.R[1], gz0 = c0[2] - G.R[2];
        // global start of every halo cell and the end of each row
        for (int h = tid; h < C.nhalo; h += blockDim.x) {
            int hx, hy, hz;
            halo_coords(h, C, hx, hy, hz);
            const uint32_t key = (uint32_t)(gx0 + hx) +
                                 (uint32_t)G.n[0] * ((uint32_t)(gy0 + hy) + (uint32_t)G.n[1] * (uint32_t)(gz0 + hz));
            raw[h] = (int)start[key];
            if (hx == C.H[0] - 1) hr_base[hy + C.H[1] * hz] = (int)start[key + 1];
        }
        __syncthreads();
        for (int r = tid; r < nhr; r += blockDim.x) {
            const int f = raw[r * C.H[0]];
            hr_first[r] = f;
            hr_base[r] -= f;  // particles in the row
        }
        __syncthreads();
        total = block_scan_smem(hr_base, nhr, wsum);
        block_scan_smem(rowpref, C.nrows, wsum);
        // staged offset of every halo cell: its row's offset plus its place in the row
        for (int h = tid; h < C.nhalo; h += blockDim.x) {
            const int r = small_div(h, C.H[0], C.invH[0]);
            lstart[h] = (uint16_t)(hr_base[r] + raw[h] - hr_first[r]);
        }
        if (tid == 0) lstart[C.nhalo] = (uint16_t)total;
        __syncthreads();  // the copy overwrites the scratch
        if (total <= C.cap) {
            // half a warp per row, consecutive lanes on consecutive particles
            const int lane = tid & 15;
            for (int r = tid >> 4; r < nhr; r += (int)blockDim.x >> 4) {
                const int j0 = hr_base[r], m = hr_base[r + 1] - j0;
                const uint32_t g0 = (uint32_t)hr_first[r];
                for (int u = lane; u < m; u += 16) {
                    const uint32_t gi = g0 + (uint32_t)u;
                    spos[j0 + u] = pos[gi];
                    if (ModeUses<MODE>::vel) svel[j0 + u] = vel[gi];
                    if (ModeUses<MODE>::rho) srho[j0 + u] = rho[gi];
                    if (MODE == 1) sid[j0 + u] = id[gi];
                }
            }
        }
        __syncthreads();
    } else {
        // halo cell counts; a ragged tile needs only ext + 2R halo cells per axis,
        // which keeps every raw coordinate within (-n, 2n) so one wrap suffices
        for (int h = tid; h < C.nhalo; h += blockDim.x) {
            int hx, hy, hz;
            halo_coords(h, C, hx, hy, hz);
            const bool inside = hx < ext[0] + 2 * G.R[0] && hy < ext[1] + 2 * G.R[1] && hz < ext[2] + 2 * G.R[2];
            const int gx = inside ? halo_cell(G, 0, c0[0], hx) : -1;
            const int gy = DIM > 1 ? halo_cell(G, 1, c0[1], hy) : 0;
            const int gz = DIM > 2 ? halo_cell(G, 2, c0[2], hz) : 0;
            uint32_t c = 0;
            if (gx >= 0 && gy >= 0 && gz >= 0) {
                const uint32_t key = (uint32_t)gx + (uint32_t)G.n[0] * ((uint32_t)gy + (uint32_t)G.n[1] * (uint32_t)gz);
                c = start[key + 1] - start[key];
            }
            // a count that does not fit 16 bits makes the tile exceed cap anyway
            lstart[h] = (uint16_t)min(c, 0xFFFFu);
        }
        __syncthreads();
        total = block_scan_smem(lstart, C.nhalo, wsum);
        block_scan_smem(rowpref, C.nrows, wsum);
        if (total <= C.cap) {
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
                // the seam shift of this halo cell (see above)
                T sh[3] = {T(0), T(0), T(0)};
                if (shifted) {
                    const int hk[3] = {hx, hy, hz};
#pragma unroll
                    for (int k = 0; k < DIM; ++k) {
                        const int raw = c0[k] - G.R[k] + hk[k];
                        if ((highk[k] && raw < G.n[k]) || (lowk[k] && raw < 0)) sh[k] = G.L[k];
                    }
                }
                for (int j = j0; j < j1; ++j) {
                    const uint32_t gi = g0 + (uint32_t)(j - j0);
                    V4<T> q = pos[gi];
                    q.x = sub_rn(q.x, sh[0]);
                    if (DIM > 1) q.y = sub_rn(q.y, sh[1]);
                    if (DIM > 2) q.z = sub_rn(q.z, sh[2]);
                    spos[j] = q;
                    if (ModeUses<MODE>::vel) svel[j] = vel[gi];
                    if (ModeUses<MODE>::rho) srho[j] = rho[gi];
                    if (MODE == 1) sid[j] = id[gi];
                }
            }
            __syncthreads();
        }
    }
    const int owned = rowpref[C.nrows];
    const bool tiled = total <= C.cap;


    for (int p = tid; p < owned; p += blockDim.x) {
        // owned row of p: the last r with rowpref[r] <= p
        int lo = 0, hi = C.nrows - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (rowpref[mid] <= p) lo = mid; else hi = mid - 1;
        }
        const int k = p - rowpref[lo];
        const uint32_t a = (uint32_t)(rowg[lo] + k);
        if (!tiled) {
            particle_global<T, DIM, MODE>(G, Ph, a, pos, vel, rho, id, start, mass, out_rho, pr_out, out_acc, cnt,
                                          fpr);
            continue;
        }
        PairAcc<T, MODE> A;
        {
            // the owned row starts at halo x = R of halo row (oy + R, oz + R)
            const int oy = lo % C.T[1], oz = lo / C.T[1];
            const int hrow = C.H[0] * ((oy + (DIM > 1 ? G.R[1] : 0)) + C.H[1] * (oz + (DIM > 2 ? G.R[2] : 0)));
            const V4<T> pa = spos[lstart[hrow + G.R[0]] + k];
            V4<T> pc = pa;  // box coordinates (adding back the shift is exact)
            if (shifted) {
                pc.x = add_rn(pa.x, orig[0]);
                if (DIM > 1) pc.y = add_rn(pa.y, orig[1]);
                if (DIM > 2) pc.z = add_rn(pa.z, orig[2]);
            }
            acc_init(A, Ph, pa, vel, rho, a);
            const bool listed = nbl.idx && p < nbl.owned_cap;
            const size_t oc = (size_t)nbl.owned_cap;
            const size_t lbase = (size_t)blockIdx.x * (size_t)(nbl.cap / 4 + 1) * oc + (size_t)p;
            if (MODE == 0 && listed) {
                // density pass: record the neighbours in walk order
                NbRec rec{nbl.idx + lbase, (uint32_t)oc, nbl.cap / 4, 0};
                if (seamless)
                    walk_tile<T, DIM, MODE, true, true>(A, G, Ph, C, c0, pa, pc, lstart, spos, svel, srho, sid, &rec);
                else
                    walk_tile<T, DIM, MODE, true, false>(A, G, Ph, C, c0, pa, pc, lstart, spos, svel, srho, sid, &rec);
                nbl.cnt[(size_t)blockIdx.x * oc + p] = rec.n <= nbl.cap ? (uint16_t)rec.n : kNbNone;
            } else if (MODE == 2 && listed && nbl.cnt[(size_t)blockIdx.x * oc + p] != kNbNone) {
                // force pass: the density pass's list of this binning, same order
                const int n = nbl.cnt[(size_t)blockIdx.x * oc + p];
                const unsigned long long *e = nbl.idx + lbase;
                const size_t st = oc;
                if (seamless)
                    read_list<T, DIM, MODE, true>(A, G, Ph, pa, spos, e, st, n);
                else
                    read_list<T, DIM, MODE, false>(A, G, Ph, pa, spos, e, st, n);
            } else if (MODE == 0) {
                // a particle the density pass does not list (rare): out of line
                if constexpr (MODE == 0) {
                    if (seamless)
                        particle_tile<T, DIM, MODE, true>(G, Ph, C, c0[0], c0[1], c0[2], pa, pc, a, lstart, spos, vel,
                                                          mass, out_rho, pr_out, out_acc);
                    else
                        particle_tile<T, DIM, MODE, false>(G, Ph, C, c0[0], c0[1], c0[2], pa, pc, a, lstart, spos, vel,
                                                           mass, out_rho, pr_out, out_acc);
                }
                continue;
            } else if (seamless) {
                walk_tile<T, DIM, MODE, false, true>(A, G, Ph, C, c0, pa, pc, lstart, spos, svel, srho, sid, nullptr);
            } else {
                walk_tile<T, DIM, MODE, false, false>(A, G, Ph, C, c0, pa, pc, lstart, spos, svel, srho, sid, nullptr);
            }
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

// Tile shape for a phase with `mean` particles per cell. The CTA's threads
// take the owned particles in turn; a tile holds about 7/8 of them per
// thread, or 1.97 (two nearly full passes) where the halo of R cells staged
// around it outweighs it (in 3D with R = 3: 8 halo cells per owned cell for
// 6^3 owned cells, 5.5 for 10 x 7 x 7), so that the halo is spread over more
// particles; in 1D and 2D, with cells of 2h (R = 1), the halo is small and
// the second pass would cost more than it saves. Its expected halo must fill at most 90 %
// of the shared-memory capacity (a tile whose halo exceeds it takes the
// global-memory walk; the 3D box's halos stay within 4 % of their mean).
// Returns false when an axis wraps fully.
template <class T>
bool plan_tiles(const Geo<T> &G, int dim, double mean, int bytes_pp, int smem_budget, TileCfg &C, size_t &smem)
{
    for (int k = 0; k < dim; ++k)
        if (G.full[k]) return false;
    int Tt[3] = {1, 1, 1};
    // owned cells for about `per_thread` owned particles per thread
    auto shape = [&](double per_thread) {
        const double target_cells = std::max(1.0, per_thread * kTileThreads / std::max(mean, 1e-6));
        const int side = std::max(1, (int)std::floor(std::pow(target_cells, 1.0 / dim) + 1e-9));
        Tt[0] = Tt[1] = Tt[2] = 1;
        for (int k = 1; k < dim; ++k) Tt[k] = std::min(side, G.n[k]);
        double rest = 1.0;
        for (int k = 1; k < dim; ++k) rest *= Tt[k];
        Tt[0] = std::max(1, std::min(G.n[0], (int)std::floor(target_cells / rest + 1e-9)));
    };
    // one pass over the owned particles (7/8 of the threads) unless the halo
    // outweighs the tile (more than 3 halo cells per owned cell, as in 3D
    // with R = 3), then two nearly full passes to spread it
    shape(0.875);
    double halo_ratio = 1.0;
    for (int k = 0; k < dim; ++k) halo_ratio *= (double)(Tt[k] + 2 * G.R[k]) / (double)Tt[k];
    if (halo_ratio > 3.0) shape(1.97);
    for (;;) {
        int H[3] = {1, 1, 1};
        long nh = 1;
        for (int k = 0; k < dim; ++k) {
            H[k] = Tt[k] + 2 * G.R[k];
            nh *= H[k];
        }
        const long nrows = (long)Tt[1] * Tt[2];
        const long nhr = (long)H[1] * H[2];
        // the halo cells' 16-bit offsets, the owned rows' prefix and starts,
        // the halo rows' starts and offsets
        const long table = lstart_bytes(nh) + 4 * (2 * nrows + 1 + 2 * nhr + 1);
        const long offset = (table + 63) / 64 * 64;
        const long cap = (smem_budget - offset) / bytes_pp;
        const double expected = mean * (double)nh;
        int kmax = 0;
        for (int k = 1; k < dim; ++k)
            if (Tt[k] > Tt[kmax]) kmax = k;
        if ((cap > 0 && expected <= 0.9 * (double)cap) || Tt[kmax] == 1) {
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
                        T *pr_out, V4<T> *out_acc, int32_t *cnt, uint64_t *fpr, double mean,
                        NbList nb = NbList{})
{
    constexpr int bpp = tile_bytes_per_particle<T, MODE>();
    const int budget = (ModeUses<MODE>::vel || ModeUses<MODE>::rho) ? 72 * 1024 : kTileSmemPos;
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
        // tile-local indices must fit the list's 15 index bits
        if (C.cap > 0x7FFF) nb = NbList{};
        k_pair_tile<T, DIM, MODE><<<blocks, kTileThreads, smem, L.stream>>>(G, Ph, C, pos, vel, rho, id, start, mass,
                                                                            out_rho, pr_out, out_acc, cnt, fpr, nb);
    } else {
        const int threads = 128;
        k_pair_global<T, DIM, MODE><<<(n + threads - 1) / threads, threads, 0, L.stream>>>(
            G, Ph, pos, vel, rho, id, start, n, mass, out_rho, pr_out, out_acc, cnt, fpr);
    }
    return cudaGetLastError();
}

template <class T, int DIM>
cudaError_t density_t(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &P, void *rho, bool gas,
                      int32_t *cnt, uint64_t *fprint, const NbList *nbl)
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
                                  static_cast<T *>(rho), pr, nullptr, nullptr, nullptr, mean,
                                  (gas && nbl) ? *nbl : NbList{});
}

template <class T, int DIM>
cudaError_t force_t(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &P, const void *rho, void *acc,
                    const NbList *nbl)
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
                                  P.start, nullptr, nullptr, static_cast<V4<T> *>(acc), nullptr, nullptr, mean,
                                  nbl ? *nbl : NbList{});
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
                           int32_t *cnt, uint64_t *fprint, const NbList *nbl)
{
    if (L.precision == TFSPH_FP64) {
        switch (L.dim) {
            case 1: return density_t<double, 1>(L, geo, phys, P, rho, gas, cnt, fprint, nbl);
            case 2: return density_t<double, 2>(L, geo, phys, P, rho, gas, cnt, fprint, nbl);
            default: return density_t<double, 3>(L, geo, phys, P, rho, gas, cnt, fprint, nbl);
        }
    }
    switch (L.dim) {
        case 1: return density_t<float, 1>(L, geo, phys, P, rho, gas, cnt, fprint, nbl);
        case 2: return density_t<float, 2>(L, geo, phys, P, rho, gas, cnt, fprint, nbl);
        default: return density_t<float, 3>(L, geo, phys, P, rho, gas, cnt, fprint, nbl);
    }
}

cudaError_t launch_force(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G, const void *rho,
                         void *acc, const NbList *nbl)
{
    if (L.precision == TFSPH_FP64) {
        switch (L.dim) {
            case 1: return force_t<double, 1>(L, geo, phys, G, rho, acc, nbl);
            case 2: return force_t<double, 2>(L, geo, phys, G, rho, acc, nbl);
            default: return force_t<double, 3>(L, geo, phys, G, rho, acc, nbl);
        }
    }
    switch (L.dim) {
        case 1: return force_t<float, 1>(L, geo, phys, G, rho, acc, nbl);
        case 2: return force_t<float, 2>(L, geo, phys, G, rho, acc, nbl);
        default: return force_t<float, 3>(L, geo, phys, G, rho, acc, nbl);
    }
}

namespace {
template <class T>
bool nblist_layout_t(const Geo<T> &G, int dim, int64_t n, int *cap, int *owned_cap, int64_t *tiles)
{
    if (n <= 0) return false;
    double ball = 4.0 * (double)G.h;  // length, area or volume within 2h
    if (dim == 2) ball = M_PI * 4.0 * (double)G.h * (double)G.h;
    if (dim == 3) ball = 4.0 / 3.0 * M_PI * 8.0 * (double)G.h * (double)G.h * (double)G.h;
    double cellv = 1.0;
    for (int k = 0; k < dim; ++k) cellv *= (double)G.w[k];
    const double mean = (double)n / (double)G.ncells;
    const double want = 1.5 * mean * ball / cellv + 16.0;
    if (want > 1024.0) return false;
    // the density pass's tiles (MODE 0 plan)
    TileCfg C{};
    size_t smem = 0;
    if (!plan_tiles(G, dim, mean, tile_bytes_per_particle<T, 0>(), kTileSmemPos, C, smem) || C.cap > 0x7FFF) return false;
    double owned = mean;
    for (int k = 0; k < dim; ++k) owned *= (double)C.T[k];
    const double cap_d = 32.0 * std::ceil(want / 32.0);
    const double oc_d = 32.0 * std::ceil((1.25 * owned + 32.0) / 32.0);
    // cap is a multiple of 32 (so of the 4 entries of a group); a particle's
    // 16-bit slots lie within cap * owned_cap + 4 of its first (32-bit offsets)
    if ((cap_d + 1.0) * oc_d >= 2147483648.0) return false;
    *cap = (int)cap_d;
    *owned_cap = (int)oc_d;
    *tiles = (int64_t)C.nt[0] * C.nt[1] * C.nt[2];
    return true;
}
}  // namespace

bool nblist_layout(const void *geo, int precision, int dim, int64_t n, int *cap, int *owned_cap, int64_t *tiles)
{
    if (precision == TFSPH_FP64)
        return nblist_layout_t(*static_cast<const Geo<double> *>(geo), dim, n, cap, owned_cap, tiles);
    return nblist_layout_t(*static_cast<const Geo<float> *>(geo), dim, n, cap, owned_cap, tiles);
}

}  // namespace tfsph
