// Per-particle steps of the binning sort shared by the single context and the
// batch: the scatter of a particle into a slot of its cell, and the rank of a
// particle inside its cell (by id), which makes the final order by (cell key,
// id) unique.
#pragma once

#include "tfsph_internal.cuh"

namespace tfsph {

// Takes one slot of cell k; a count that is already zero or a slot past the
// end means the counts and keys disagree: flagged, nothing written.
__device__ __forceinline__ void scatter_one(uint32_t i, const uint32_t *__restrict__ key,
                                            const uint32_t *__restrict__ id, uint32_t *__restrict__ cnt,
                                            const uint32_t *__restrict__ start, uint32_t *__restrict__ src,
                                            uint32_t *__restrict__ tid, uint32_t n, int *err)
{
    const uint32_t k = key[i];
    const uint32_t old = atomicSub(&cnt[k], 1u);
    const uint32_t slot = start[k] + old - 1u;
    if (old == 0u || slot >= n) {
        atomicAdd(&cnt[k], 1u);
        atomicOr(err, kErrInternal);
        return;
    }
    src[slot] = i;
    tid[slot] = id[i] & kIdMask;
}

// Runs of consecutive lanes of a full warp that hold the same counter take
// it with one atomic, issued by the run's first lane. After the previous
// sort, the particles of a cell sit next to each other in storage, so a cell
// holding several particles of a phase costs one atomic per warp instead of
// one per particle. Returns the run's first lane and sets *m to its length
// and *full to whether the whole warp took part (if not, each lane is a run
// of its own).
__device__ __forceinline__ int counter_run(const uint32_t *c, uint32_t *m, bool *full)
{
    const unsigned act = __activemask();
    const int lane = (int)(threadIdx.x & 31u);
    *full = act == 0xffffffffu;
    if (!*full) {
        *m = 1u;
        return lane;
    }
    const unsigned long long a = (unsigned long long)c;
    const unsigned long long prev = __shfl_up_sync(0xffffffffu, a, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != a);
    const unsigned le = lane == 31 ? 0xffffffffu : ((1u << (lane + 1)) - 1u);
    const int first = 31 - __clz(heads & le);
    const unsigned after = heads & ~le;
    const int end = after ? __ffs(after) - 1 : 32;
    *m = (uint32_t)(end - first);
    return first;
}

__device__ __forceinline__ void count_add_agg(uint32_t *c)
{
    uint32_t m;
    bool full;
    const int first = counter_run(c, &m, &full);
    if ((int)(threadIdx.x & 31u) == first) atomicAdd(c, m);
}

// scatter_one with the atomics of a run of lanes on one counter combined:
// each lane receives the value a lone atomicSub of its own would have
// returned, in lane order within the run.
__device__ __forceinline__ void scatter_one_agg(uint32_t i, const uint32_t *__restrict__ key,
                                                const uint32_t *__restrict__ id, uint32_t *__restrict__ cnt,
                                                const uint32_t *__restrict__ start, uint32_t *__restrict__ src,
                                                uint32_t *__restrict__ tid, uint32_t n, int *err)
{
    const uint32_t k = key[i];
    uint32_t *c = &cnt[k];
    uint32_t m;
    bool full;
    const int first = counter_run(c, &m, &full);
    const int lane = (int)(threadIdx.x & 31u);
    const uint32_t rank = (uint32_t)(lane - first);
    uint32_t old = 0;
    if (rank == 0u) old = atomicSub(c, m);
    if (full) old = __shfl_sync(0xffffffffu, old, first);
    const uint32_t mine = old - rank;  // this lane's share of the count
    const uint32_t slot = start[k] + mine - 1u;
    if (old <= rank || slot >= n) {
        atomicAdd(c, 1u);
        atomicOr(err, kErrInternal);
        return;
    }
    src[slot] = i;
    tid[slot] = id[i] & kIdMask;
}

template <class T>
__device__ __forceinline__ void rank_move(uint32_t s, const uint32_t *__restrict__ key,
                                          const uint32_t *__restrict__ start, const uint32_t *__restrict__ src,
                                          const uint32_t *__restrict__ tid, const V4<T> *__restrict__ pos,
                                          const V4<T> *__restrict__ vel, const uint32_t *__restrict__ id,
                                          V4<T> *__restrict__ opos, V4<T> *__restrict__ ovel,
                                          uint32_t *__restrict__ oid, uint32_t n, int *err)
{
    const uint32_t i = src[s];
    if (i >= n) {  // a slot the scatter did not fill (flagged there too)
        atomicOr(err, kErrInternal);
        return;
    }
    const uint32_t k = key[i];
    const uint32_t b = start[k], e = start[k + 1];
    uint32_t d = b;
    if (e - b > 1) {
        const uint32_t mine = tid[s];
        for (uint32_t t = b; t < e; ++t) d += tid[t] < mine ? 1u : 0u;
    }
    if (d >= e) {
        atomicOr(err, kErrInternal);
        return;
    }
    opos[d] = pos[i];
    ovel[d] = vel[i];
    oid[d] = id[i];
}

}  // namespace tfsph
