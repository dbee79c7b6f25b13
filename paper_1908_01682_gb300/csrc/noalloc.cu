// Cell ranges from cell keys without any device allocation.
//
// Variant of the library's binning count + scan for callers that cannot
// allocate device memory: the per-cell counters and the scan's block totals
// live in one file-scope static device array, set aside when the library is
// loaded and kept by every GPU that loads it until the process exits.
#include <cstdio>
#include <mutex>

#include "tfsph_internal.cuh"

namespace {

constexpr uint32_t kMaxCells = 1u << 21;          // 2,097,152 cells
constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr uint32_t kTile = kThreads * kItems;      // cells per scan block
constexpr uint32_t kMaxBlocks = (kMaxCells + kTile - 1) / kTile;
constexpr uint32_t kScratchWords = kMaxCells + kMaxBlocks;  // counters, then block totals (8 MiB + 4 KiB)

static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current (the symbol's name is only a host-side stand-in).
std::mutex g_setup_mutex;
constexpr int kMaxDevices = 64;
uint32_t *g_scratch_ptr[kMaxDevices] = {nullptr};

int noalloc_fail(int code, const char *msg)
{
    tfsph::set_unbound_error(msg);  // reported by tfsph_last_error(NULL)
    return code;
}

__global__ void k_na_count(const uint32_t *__restrict__ keys, int n, uint32_t n_cells, uint32_t *__restrict__ cnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = keys[i];
    if (k < n_cells) atomicAdd(&cnt[k], 1u);  // keys outside [0, n_cells) are not counted
}

__device__ __forceinline__ uint32_t na_block_scan(uint32_t v, uint32_t &excl)
{
    __shared__ uint32_t warp_tot[kThreads / 32];
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
        uint32_t t = lane < kThreads / 32 ? warp_tot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kThreads / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    excl = (wid > 0 ? warp_tot[wid - 1] : 0u) + x - v;
    const uint32_t total = warp_tot[kThreads / 32 - 1];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(kThreads)
k_na_reduce(const uint32_t *__restrict__ cnt, uint32_t n_cells, uint32_t *__restrict__ bsum)
{
    const uint32_t base = blockIdx.x * kTile + threadIdx.x * kItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k)
        if (base + k < n_cells) s += cnt[base + k];
    uint32_t excl;
    const uint32_t tot = na_block_scan(s, excl);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kThreads) k_na_top(uint32_t *__restrict__ bsum, uint32_t nblk)
{
    uint32_t carry = 0;
    for (uint32_t base = 0; base < nblk; base += kThreads) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nblk ? bsum[i] : 0u;
        uint32_t excl;
        const uint32_t tot = na_block_scan(v, excl);
        if (i < nblk) bsum[i] = carry + excl;
        carry += tot;
    }
}

__global__ void __launch_bounds__(kThreads)
k_na_down(const uint32_t *__restrict__ cnt, uint32_t n_cells, const uint32_t *__restrict__ bsum,
          uint32_t *__restrict__ starts)
{
    const uint32_t base = blockIdx.x * kTile + threadIdx.x * kItems;
    uint32_t v[kItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        v[k] = base + k < n_cells ? cnt[base + k] : 0u;
        s += v[k];
    }
    uint32_t excl;
    na_block_scan(s, excl);
    uint32_t run = bsum[blockIdx.x] + excl;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (base + k < n_cells) starts[base + k] = run;
        run += v[k];
    }
    // the block holding the last cell writes the total after it
    if (base <= n_cells - 1 && n_cells - 1 < base + kItems) starts[n_cells] = run;
}

}  // namespace

extern "C" int tfsph_cell_ranges_noalloc(const uint32_t *keys, int64_t n, uint32_t n_cells, uint32_t *starts,
                                         void *stream)
{
    if (n_cells == 0 || n_cells > kMaxCells)
        return noalloc_fail(TFSPH_E_INVALID_ARG, "n_cells must be in [1, 2097152] (the static scratch holds 2^21 cell counters)");
    if (n < 0 || n >= ((int64_t)1 << 31)) return noalloc_fail(TFSPH_E_INVALID_ARG, "n must be in [0, 2^31)");
    if (!starts || (n > 0 && !keys)) return noalloc_fail(TFSPH_E_INVALID_ARG, "NULL keys or starts");
    // an error left by an earlier, unrelated call stays the caller's: report
    // it without clearing it, so the status below only ever describes this
    // call's own launches
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return noalloc_fail(TFSPH_E_CUDA, "a CUDA error from an earlier call is pending");
    int dev = -1;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(TFSPH_E_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(TFSPH_E_INVALID_ARG, "device ordinal out of range");
    uint32_t *scratch;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) return noalloc_fail(TFSPH_E_CUDA, "cudaGetSymbolAddress of the static scratch failed");
            g_scratch_ptr[dev] = static_cast<uint32_t *>(ptr);
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t *cnt = scratch;
    uint32_t *bsum = scratch + kMaxCells;
    const uint32_t nblk = (n_cells + kTile - 1) / kTile;
    // the scratch keeps the previous call's contents: the counters start from zero
    e = cudaMemsetAsync(cnt, 0, (size_t)n_cells * sizeof(uint32_t), s);
    if (e != cudaSuccess) return noalloc_fail(TFSPH_E_CUDA, cudaGetErrorString(e));
    if (n > 0) k_na_count<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(keys, (int)n, n_cells, cnt);
    k_na_reduce<<<nblk, kThreads, 0, s>>>(cnt, n_cells, bsum);
    k_na_top<<<1, kThreads, 0, s>>>(bsum, nblk);
    k_na_down<<<nblk, kThreads, 0, s>>>(cnt, n_cells, bsum, starts);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(TFSPH_E_CUDA, cudaGetErrorString(e));
    return TFSPH_OK;
}
