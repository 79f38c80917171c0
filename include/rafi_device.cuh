/*
 * rafi_device.cuh -- device side of the forwarding interface (Sec. 3.3).
 *
 * Header-only CUDA helpers over rf_device_queues (rafi.h) for kernels that
 * read incoming work and forward outgoing work:
 *
 *   rf::numIncoming(q)         items incoming over all ranks
 *   rf::numIncoming(q, rank)   items incoming for one rank
 *   rf::getIncoming<T>(q, i)   read incoming item i (any thread, any order)
 *   rf::rankOf(q, i)           rank whose segment holds incoming item i
 *   rf::forward(q, item, dst)  append item for rank dst (emitOutgoing); one
 *                              atomicAdd per group of converged lanes
 *   rf::BlockForward<B>        block-cooperative forward: one atomicAdd per block
 *
 * Items are trivially copyable structs of q.itemBytes bytes, a multiple of 16;
 * they move as 16-byte vectors.  Sending to one's own rank is valid; an emit
 * at or past capacity is dropped and reported by the next exchange (Sec. 3.3).
 */
#ifndef RAFI_DEVICE_CUH
#define RAFI_DEVICE_CUH

#include <cooperative_groups.h>

#include "rafi.h"

namespace rf {

__device__ __forceinline__ uint32_t numIncoming(const rf_device_queues &q)
{
    return q.inOffset[q.numRanks];
}

__device__ __forceinline__ uint32_t numIncoming(const rf_device_queues &q, int32_t rank)
{
    return q.inOffset[rank + 1] - q.inOffset[rank];
}

template <class T>
__device__ __forceinline__ T getIncoming(const rf_device_queues &q, uint32_t i)
{
    static_assert(sizeof(T) % 16 == 0, "forwarded items are multiples of 16 bytes");
    T v;
    const uint4 *src = reinterpret_cast<const uint4 *>(q.in) + (size_t)i * (sizeof(T) / 16);
    uint4 *dst = reinterpret_cast<uint4 *>(&v);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(T) / 16); ++k) dst[k] = src[k];
    return v;
}

/* Largest r with inOffset[r] <= i (segments are sorted; empty ranks skipped). */
__device__ __forceinline__ int32_t rankOf(const uint32_t *offsets, int32_t numRanks, uint32_t i)
{
    int32_t lo = 0, hi = numRanks; /* invariant: offsets[lo] <= i < offsets[hi] */
    while (hi - lo > 1) {
        int32_t mid = (lo + hi) >> 1;
        if (offsets[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int32_t rankOf(const rf_device_queues &q, uint32_t i)
{
    return rankOf(q.inOffset, q.numRanks, i);
}

template <class T>
__device__ __forceinline__ void storeItem(const rf_device_queues &q, unsigned long long slot, const T &item,
                                          int32_t dst)
{
    uint4 *o = reinterpret_cast<uint4 *>(q.out) + (size_t)slot * (sizeof(T) / 16);
    const uint4 *s = reinterpret_cast<const uint4 *>(&item);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(T) / 16); ++k) o[k] = s[k];
    q.dest[slot] = dst;
}

/* emitOutgoing(ray, dest) (Sec. 3.3 / 4.1): atomically append item for rank
 * dst.  The lanes that call it together share one atomicAdd.  Returns false
 * if the item was dropped for lack of capacity. */
template <class T>
__device__ __forceinline__ bool forward(const rf_device_queues &q, const T &item, int32_t dst)
{
    static_assert(sizeof(T) % 16 == 0, "forwarded items are multiples of 16 bytes");
    namespace cg = cooperative_groups;
    cg::coalesced_group g = cg::coalesced_threads();
    unsigned long long base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(q.outCount, (unsigned long long)g.size());
    base = g.shfl(base, 0);
    unsigned long long slot = base + g.thread_rank();
    if (slot >= q.capacity) return false;
    storeItem(q, slot, item, dst);
    return true;
}

template <class T>
__device__ __forceinline__ bool emitOutgoing(const rf_device_queues &q, const T &item, int32_t dst)
{
    return forward(q, item, dst);
}

/* Block-cooperative append: every thread of the (1-D, BLOCK-thread) block
 * calls reserve() with its flag; it returns the slot for a flagged thread.
 * One atomicAdd on counter per block. */
template <int BLOCK>
struct BlockAppend {
    static_assert(BLOCK % 32 == 0 && BLOCK <= 1024, "block of whole warps");
    struct Storage {
        unsigned warpBase[BLOCK / 32];
        unsigned long long blockBase;
    };
    __device__ __forceinline__ static unsigned long long reserve(Storage &s, unsigned long long *counter,
                                                                 bool flag)
    {
        const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
        const unsigned ballot = __ballot_sync(0xFFFFFFFFu, flag);
        const unsigned below = __popc(ballot & ((1u << lane) - 1u));
        if (lane == 0) s.warpBase[warp] = __popc(ballot);
        __syncthreads();
        if (threadIdx.x < 32) {
            unsigned v = threadIdx.x < BLOCK / 32 ? s.warpBase[threadIdx.x] : 0u;
            unsigned incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if ((int)threadIdx.x >= o) incl += t;
            }
            if (threadIdx.x < BLOCK / 32) s.warpBase[threadIdx.x] = incl - v;
            if (threadIdx.x == 31) s.blockBase = incl ? atomicAdd(counter, (unsigned long long)incl) : 0ull;
        }
        __syncthreads();
        unsigned long long slot = s.blockBase + s.warpBase[warp] + below;
        __syncthreads(); /* storage may be reused right after */
        return slot;
    }
};

/* Block-cooperative forward: all BLOCK threads call it; threads with
 * flag == false take no slot.  Returns false for a flagged item that was
 * dropped for lack of capacity. */
template <int BLOCK, class T>
__device__ __forceinline__ bool BlockForward(typename BlockAppend<BLOCK>::Storage &s, const rf_device_queues &q,
                                             const T &item, int32_t dst, bool flag)
{
    unsigned long long slot = BlockAppend<BLOCK>::reserve(s, q.outCount, flag);
    if (!flag || slot >= q.capacity) return !flag;
    storeItem(q, slot, item, dst);
    return true;
}

} // namespace rf

#endif /* RAFI_DEVICE_CUH */
