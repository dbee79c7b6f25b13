// Internal declarations shared by the CUDA translation units of libtfsph.
//
// Data layout in HBM (per phase, structure of arrays, double-buffered for the
// gather into cell order):
//   pos[2]  : V4<T> per particle. Gas: (x, y, z, p/rho^2 after the density
//             pass); dust: (x, y, z, 0).
//   vel[2]  : V4<T> per particle. Gas: (vx, vy, vz, e); dust: (ux, uy, uz, t_stop).
//   id[2]   : uint32 particle id; bit 31 marks a frozen (wall) gas particle.
//   key     : uint32 cell key of the particle in each storage slot, written by
//             the update of the previous step (or at set-up).
//   count   : uint32 per cell, zero between steps (the scatter counts it down).
//   start   : uint32 per cell + 1, first storage slot of each cell.
// Gas only: rho (T) and acc (V4<T>: ax, ay, az, de/dt).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "tfsph.h"

namespace tfsph {

constexpr uint32_t kIdMask = 0x7fffffffu;
constexpr uint32_t kFrozenBit = 0x80000000u;

// Device error word bits (set by kernels, read by tfsph_sync).
constexpr int kErrBadTstop = 1;
constexpr int kErrInternal = 2;
constexpr int kErrTimeout = 4;   // a bounded device-side wait ran out

struct alignas(32) double4a {
    double x, y, z, w;
};

template <class T> struct Vec4Of;
template <> struct Vec4Of<float> { using type = float4; };
template <> struct Vec4Of<double> { using type = double4a; };
template <class T> using V4 = typename Vec4Of<T>::type;

// IEEE operations with explicit round-to-nearest, so the compiler cannot fuse
// them; used wherever a floating-point result decides an integer (cell keys,
// neighbour membership) and must match the checker's plain arithmetic.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Grid geometry and neighbour-search constants, built on the host in double
// and rounded once to T.
template <class T> struct Geo {
    int dim;
    int n[3];      // cells per axis
    int R[3];      // reach in cells per axis
    int per[3];    // periodic axis
    int full[3];   // periodic axis whose window covers every cell
    T lo[3];
    T inv_w[3];    // cells per unit length, (T)(n / L)
    T w[3];        // cell edge
    T L[3];        // box edge (periodic axes)
    T halfL[3];
    T h2x4;        // (T)(4 h^2): neighbour iff r^2 < h2x4
    T lim2;        // squared pruning radius for candidate cells (2h plus margin)
    T wnorm;       // sigma_d / h^d
    T fnorm;       // sigma_d / h^(d+2): (1/r) dW/dr = fnorm * g(q)
    T inv_h;
    T h;
    uint32_t ncells;
    // exact cell index (cell_key): per axis, n + 1 device values; thr[d][i]
    // (0 < i < n) is the smallest T value at or above the face lo + i L / n
    // between cells i - 1 and i (real arithmetic, L = hi - lo in binary64),
    // so that for a stored coordinate x, x >= face i exactly when
    // x >= thr[d][i]; entries 0 and n are -inf and +inf (not read).
    const T *thr[3];
    // 1 when the rounded estimate is itself exact along the axis: lo = 0 and
    // n / L a power of two, so x - lo and the scaling by n / L are exact in T
    int est_exact[3];
};

// Fills thr[0..n] for one axis (host): the smallest T value at or above
// each face lo + i (hi - lo)/n, each settled by the exact sign of
// (x - lo) n - i L. Defined in params.cu for T = float and double.
template <class T> void face_thresholds(double lo, double hi, int n, T *thr);

template <class T> struct Phys {
    T m_g, m_d;
    T cs, cs2;
    T gm1, gamma;     // gamma - 1, gamma
    T av_alpha, av_beta;
    T eta2;           // 0.01 h^2
    T h;
    T wnorm4;         // sigma_d / h^d / 4: the density sums accumulate 4 W / (sigma_d / h^d)
    T mfnorm;         // m_g sigma_d / h^(d+2): the isothermal force sums accumulate (1/r) dW/dr / fnorm
    T hm075;          // -3/4 h
    int eos;
    int av;
};

struct PhaseBufs {
    int64_t n = 0;
    void *pos[2] = {nullptr, nullptr};
    void *vel[2] = {nullptr, nullptr};
    uint32_t *id[2] = {nullptr, nullptr};
    uint32_t *key = nullptr;
    uint32_t *count = nullptr;
    uint32_t *start = nullptr;
    uint32_t *tmp_src = nullptr;
    uint32_t *tmp_id = nullptr;
    int cur = 0;
};

// Compact neighbour list of the gas pair sums, written by the tiled density
// pass and read by the tiled force pass of the same binning (both passes use
// the same tiles and visit the owned particles of a tile in the same order).
// An entry is the tile-local (shared-memory) index of a neighbour, bit 15
// set for a pair across a periodic seam. A particle's entries, in walk
// order, are packed four to a 64-bit group (entry k at bits 16 (k mod 4) of
// group k / 4); for owned particle p < owned_cap of tile t, group g is
// idx[(t * (cap / 4 + 1) + g) * owned_cap + p], so a warp's accesses are
// contiguous; group cap / 4 of each tile is a spare that takes (and drops)
// the groups beyond cap (a multiple of 4) entries. cnt[t * owned_cap + p] is
// the number of entries, or kNbNone when the particle has more than cap
// neighbours; such particles (and p >= owned_cap) walk their candidates again.
struct NbList {
    unsigned long long *idx = nullptr;
    uint16_t *cnt = nullptr;
    int cap = 0;
    int owned_cap = 0;
};
constexpr uint16_t kNbNone = 0xFFFFu;
constexpr uint16_t kNbSeam = 0x8000u;

// Scan partials: blocks of kScanTile cells.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;  // the scan kernels move them as two 16-byte words
constexpr int kScanTile = kScanThreads * kScanItems;

// Cell-update CTA: one thread per cell in phase 1.
constexpr int kCellsPerCta = 128;

// ---------------------------------------------------------------------------
// Launchers (host functions), grouped by translation unit.
// ---------------------------------------------------------------------------
struct LaunchCtx {
    cudaStream_t stream;
    int precision;   // TFSPH_FP32 / TFSPH_FP64
    int dim;
    int *d_err;      // device error word
    cudaEvent_t *ev; // optional phase events: launch_bin records ev[1..4]
};

// bin.cu
cudaError_t launch_keys(const LaunchCtx &L, const void *geo, const PhaseBufs &P);
cudaError_t launch_bin(const LaunchCtx &L, const void *geo, PhaseBufs &G, PhaseBufs &D,
                       uint32_t *bsum, int64_t nblk);
cudaError_t launch_pack(const LaunchCtx &L, PhaseBufs &P, const void *const *src, int ncomp_v,
                        const uint8_t *frozen, bool is_gas);
cudaError_t launch_unpack(const LaunchCtx &L, const PhaseBufs &P, int what, void *out, int order,
                          const void *aux);
cudaError_t launch_set_tstop(const LaunchCtx &L, PhaseBufs &D, const void *t_stop);
cudaError_t launch_check(const LaunchCtx &L, const void *geo, const PhaseBufs &P, int is_gas,
                         int *flags);
cudaError_t launch_max_speed(const LaunchCtx &L, const void *phys, const PhaseBufs &G,
                             void *partials, int nblk, void *result);
cudaError_t launch_debug_keys(const LaunchCtx &L, const void *geo, const PhaseBufs &P, uint32_t *out);
// One launch each for all adjoint arrays of a step: into storage order (and
// lts cleared), and back to id order.
cudaError_t launch_lam_gather_all(const LaunchCtx &L, const PhaseBufs &G, const PhaseBufs &D, const void *lgx,
                                  const void *lgv, const void *ldx, const void *ldu, void *gx4, void *gv4, void *dx4,
                                  void *du4, void *lts);
cudaError_t launch_lam_scatter_all(const LaunchCtx &L, const PhaseBufs &G, const PhaseBufs &D, const void *gx4,
                                   const void *out, const void *gv4, const void *du4, const void *lts, void *lgx,
                                   void *lgv, void *ldu, void *lt);
cudaError_t launch_lamq_to_lamrho(const LaunchCtx &L, const PhaseBufs &P, const void *lq, const void *rho, double cs2,
                                  void *lrho);

// sph.cu. The density pass writes *nbl when given (gas only), the force pass
// reads it when given (it must come from the density pass of this binning).
cudaError_t launch_density(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &P,
                           void *rho, bool gas, int32_t *cnt, uint64_t *fprint, const NbList *nbl = nullptr);
cudaError_t launch_force(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G,
                         const void *rho, void *acc, const NbList *nbl = nullptr);
// Shape of the neighbour list for a gas phase of n particles: entries per
// particle (about 1.5 times the expected neighbour count, a multiple of 32),
// owned particles per tile with a list, and tiles; false when the density
// pass of this geometry is not tiled or its tiles cannot index a list.
bool nblist_layout(const void *geo, int precision, int dim, int64_t n, int *cap, int *owned_cap, int64_t *tiles);
cudaError_t launch_force_adjoint(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G,
                                 const void *lamA, void *out);
cudaError_t launch_density_adjoint(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G,
                                   const void *lamrho, void *inout);

// tfsph_api.cu: message for tfsph_last_error(NULL) from calls without a context
void set_unbound_error(const char *msg);

// params.cu: checks of one parameter set with its particle counts (a
// TFSPH_E_* code, the reason in why), and its cell grid (cells per axis;
// returns the cell count; validate_params bounds it by 1e9).
int validate_params(const tfsph_params *p, int64_t ng, int64_t nd, std::string &why);
uint32_t cell_grid(const tfsph_params &p, int ncell[3]);

// Grid geometry and physical constants of a parameter set, computed in double
// and rounded once to T. The pruning radius is 2h plus a margin covering the
// rounding of cell coordinates and of r^2, so no neighbour is ever pruned.
template <class T>
void make_geo_phys(const tfsph_params &p, const int ncell[3], uint32_t ncells, Geo<T> &G, Phys<T> &Ph)
{
    G = Geo<T>{};
    G.dim = p.dim;
    const double u = sizeof(T) == 4 ? 0x1p-24 : 0x1p-53;
    double span = 0.0;
    for (int d = 0; d < p.dim; ++d) span = fmax(span, fmax(fabs(p.lo[d]), fabs(p.hi[d])) + (p.hi[d] - p.lo[d]));
    const double margin = 8.0 * u * span + 16.0 * u * 2.0 * p.h;
    const double reach = 2.0 * p.h + margin;
    for (int d = 0; d < 3; ++d) {
        if (d >= p.dim) {
            G.n[d] = 1;
            G.R[d] = 0;
            G.per[d] = 0;
            G.full[d] = 0;
            G.lo[d] = T(0);
            G.inv_w[d] = T(0);
            G.w[d] = T(1);
            G.L[d] = T(1);
            G.halfL[d] = T(0.5);
            G.thr[d] = nullptr;
            G.est_exact[d] = 1;
            continue;
        }
        const double L = p.hi[d] - p.lo[d];
        const int n = ncell[d];
        const double w = L / (double)n;
        G.n[d] = n;
        G.R[d] = (int)floor(reach / w) + 1;
        G.per[d] = p.periodic[d] ? 1 : 0;
        G.full[d] = (G.per[d] && 2 * G.R[d] + 1 >= n) ? 1 : 0;
        G.lo[d] = T(p.lo[d]);
        G.inv_w[d] = T((double)n / L);
        G.w[d] = T(w);
        G.L[d] = T(L);
        G.halfL[d] = T(0.5 * L);
        G.thr[d] = nullptr;  // set by the owner of the device table
        int ex = 0;
        const double mant = frexp((double)n / L, &ex);
        G.est_exact[d] = (p.lo[d] == 0.0 && mant == 0.5 && (double)T((double)n / L) == (double)n / L) ? 1 : 0;
    }
    G.h2x4 = T(4.0 * p.h * p.h);
    G.lim2 = T(reach * reach * (1.0 + 16.0 * u));
    const double sigma = p.dim == 1 ? 2.0 / 3.0 : (p.dim == 2 ? 10.0 / (7.0 * M_PI) : 1.0 / M_PI);
    G.wnorm = T(sigma / pow(p.h, p.dim));
    G.fnorm = T(sigma / pow(p.h, p.dim + 2));
    G.inv_h = T(1.0 / p.h);
    G.h = T(p.h);
    G.ncells = ncells;

    Ph = Phys<T>{};
    Ph.m_g = T(p.m_gas);
    Ph.m_d = T(p.m_dust);
    Ph.cs = T(p.cs);
    Ph.cs2 = T(p.cs * p.cs);
    Ph.gm1 = T(p.gamma - 1.0);
    Ph.gamma = T(p.gamma);
    Ph.av_alpha = T(p.av_alpha);
    Ph.av_beta = T(p.av_beta);
    Ph.eta2 = T(0.01 * p.h * p.h);
    Ph.h = T(p.h);
    Ph.wnorm4 = T(0.25 * sigma / pow(p.h, p.dim));
    Ph.mfnorm = T(p.m_gas * sigma / pow(p.h, p.dim + 2));
    Ph.hm075 = T(-0.75 * p.h);
    Ph.eos = p.eos;
    Ph.av = (p.av_alpha > 0.0 || p.av_beta > 0.0) ? 1 : 0;
}

// drag.cu
struct StepArgs {
    double tau;
    double g[3];
    int tstar_mode;
    int cell_acc;
    int has_frozen;
};
cudaError_t launch_cell_update(const LaunchCtx &L, const void *geo, const void *phys,
                               PhaseBufs &G, PhaseBufs &D, const void *acc, const StepArgs &S);
// xdrag.cu: the ISPH or MK drag and particle update (scheme TFSPH_DRAG_ISPH |
// TFSPH_DRAG_MK) after binning, gas and dust densities and the gas pressure
// force. Scratch per particle: g4, d4, d4b (V4) and g1 (T).
struct XDragBufs {
    void *g4 = nullptr, *g1 = nullptr, *d4 = nullptr, *d4b = nullptr;
};
cudaError_t launch_xdrag(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G, PhaseBufs &D,
                         const void *rho_g, const void *rho_d, const void *acc, const XDragBufs &B,
                         const StepArgs &S, int scheme);
cudaError_t launch_cell_adjoint(const LaunchCtx &L, const void *geo, const void *phys, PhaseBufs &G, PhaseBufs &D,
                                const void *acc, const StepArgs &S, const void *lgx, void *lgv, const void *ldx,
                                void *ldu, void *lA, void *lts);

// ---------------------------------------------------------------------------
// Device helpers shared by the kernels.
// ---------------------------------------------------------------------------
// Rounded cell coordinate t = fl(fl(x - lo) inv) and its floor, clamped to
// [0, n - 1] (negative or NaN: 0). Places the candidate window of the pair
// walks, and starts the exact index (exact_cell), within one cell of it.
template <class T> __device__ __forceinline__ int axis_cell(T x, T lo, T inv, int n, T &t)
{
    t = mul_rn(sub_rn(x, lo), inv);
    T f = floor(t);
    int i;
    if (!(f >= T(0))) i = 0;          // negative or NaN
    else if (f >= T(n)) i = n - 1;
    else i = (int)f;
    return i;
}

// Cell index along axis d, exact: floor((x - lo) n / L) over the reals for
// the stored coordinate x, lo and L = hi - lo in binary64, clamped to
// [0, n - 1], NaN to 0 (Sec. 2.3: membership of the disjoint volumes). The
// rounded estimate is within one cell of it; the face thresholds move it to
// the exact index (two moves at most either way, whatever happens).
template <class T, bool EST = false> __device__ __forceinline__ int exact_cell(const Geo<T> &G, int d, T x)
{
    T t;
    const int n = G.n[d];
    int i = axis_cell(x, G.lo[d], G.inv_w[d], n, t);
    if (EST || G.est_exact[d]) return i;
    if (!(x == x)) return 0;
    const T *thr = G.thr[d];
    if (i > 0 && x < __ldg(&thr[i])) {
        --i;
        if (i > 0 && x < __ldg(&thr[i])) --i;
    } else if (i < n - 1 && !(x < __ldg(&thr[i + 1]))) {
        ++i;
        if (i < n - 1 && !(x < __ldg(&thr[i + 1]))) ++i;
    }
    return i;
}

// Cell key, exact per axis; key = ix + nx (iy + ny iz). EST: the caller
// knows that every axis has est_exact set (the table is not read).
template <class T, int DIM, bool EST = false>
__device__ __forceinline__ uint32_t cell_key(const Geo<T> &G, T x, T y, T z)
{
    const int ix = exact_cell<T, EST>(G, 0, x);
    const int iy = DIM > 1 ? exact_cell<T, EST>(G, 1, y) : 0;
    const int iz = DIM > 2 ? exact_cell<T, EST>(G, 2, z) : 0;
    return (uint32_t)ix + (uint32_t)G.n[0] * ((uint32_t)iy + (uint32_t)G.n[1] * (uint32_t)iz);
}

// Minimum-image displacement along one axis, in the order the checker uses.
template <class T> __device__ __forceinline__ T min_image(T d, int per, T L, T half)
{
    if (per) {
        if (d > half) d = sub_rn(d, L);
        else if (d < -half) d = add_rn(d, L);
    }
    return d;
}

// Periodic image of x in [lo, lo + L).
template <class T> __device__ __forceinline__ T wrap_periodic(T x, T lo, T L)
{
    T y = x - lo;
    y -= L * floor(y / L);
    T r = lo + y;
    if (r >= lo + L) r = lo;
    if (r < lo) r = lo;
    return r;
}

// Value arithmetic (never a decision): hardware approximations in binary32
// (sqrt.approx / rsqrt.approx, relative error below 2^-22; fast division,
// 2 ulp), IEEE operations in binary64.
__device__ __forceinline__ float approx_sqrt(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double approx_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float approx_rsqrt(float x)
{
    float r;
    asm("rsqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double approx_rsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float approx_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double approx_div(double a, double b) { return a / b; }

// Square root and reciprocal square root of a pair's r^2, with subnormal
// inputs flushed to zero (no rescaling of subnormal inputs, which the forms
// above carry): the pair sums treat r^2 below pair_r2_min() (the smallest
// normal binary32 number; the smallest subnormal in binary64) as a zero
// displacement.
__device__ __forceinline__ float pair_sqrt(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double pair_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float pair_rsqrt(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double pair_rsqrt(double x) { return 1.0 / sqrt(x); }
template <class T> __device__ __forceinline__ T pair_r2_min();
template <> __device__ __forceinline__ float pair_r2_min<float>() { return 1.17549435e-38f; }
template <> __device__ __forceinline__ double pair_r2_min<double>() { return 4.9406564584124654e-324; }

// Fused multiply-add with one rounding, for the neighbour decision r^2.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// M4 cubic spline (support 2h), branch free on q in [0, 2):
//   W = wnorm * (q < 1 ? 1 - 3/2 q^2 + 3/4 q^3 : 1/4 (2 - q)^3)
//   (1/r) dW/dr = fnorm * (q < 1 ? -3 + 9/4 q : -3/4 (2 - q)^2 / q)
template <class T> __device__ __forceinline__ T kernel_w(const Geo<T> &G, T q)
{
    const T a = fmax(T(2) - q, T(0));
    const T inner = T(1) + q * q * (T(-1.5) + T(0.75) * q);
    const T outer = T(0.25) * a * a * a;
    return G.wnorm * (q < T(1) ? inner : outer);
}

// 4 W / (sigma_d / h^d): the density sums add this and scale once at the end
//   (q < 1 ? 4 - 6 q^2 + 3 q^3 : (2 - q)^3)
template <class T> __device__ __forceinline__ T kernel_w4(T q)
{
    const T a = fmax(T(2) - q, T(0));
    const T inner = T(4) + q * q * (T(-6) + T(3) * q);
    return q < T(1) ? inner : a * a * a;
}

template <class T> __device__ __forceinline__ T kernel_f(const Geo<T> &G, T q, T inv_q)
{
    const T a = fmax(T(2) - q, T(0));
    return G.fnorm * (q < T(1) ? T(-3) + T(2.25) * q : T(-0.75) * a * a * inv_q);
}

// d/dr of (1/r) dW/dr:
//   fnorm / h * (q < 1 ? 9/4 : 3/4 (2 - q)(2 + q) / q^2)
template <class T> __device__ __forceinline__ T kernel_fprime(const Geo<T> &G, T q, T inv_q)
{
    const T a = fmax(T(2) - q, T(0));
    return G.fnorm * G.inv_h * (q < T(1) ? T(2.25) : T(0.75) * a * (q + T(2)) * inv_q * inv_q);
}

}  // namespace tfsph
