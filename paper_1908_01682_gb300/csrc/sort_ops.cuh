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
