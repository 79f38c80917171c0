// Batched form of the forwarding loop: every round of "work, then exchange"
// in one persistent cooperative kernel, with no host round trip per round.
//
// The plain loop (Sec. 5.1's "alternate between the render kernel and
// forwardRays until no ray is left") launches a work kernel and the exchange
// kernels per round and reads the active count back on the host.  Here all
// CTAs of one cooperative launch stay resident and run the rounds
// themselves:
//
//   phase 1  the workload's step over the incoming queue, written back to
//            the same slots of the out-queue with each item's destination
//            (the paper's first single-array queue, Sec. 3.2): tile by tile
//            over a contiguous range per CTA, or in dynamically handed-out
//            chunks for policies with long, uneven steps; then each CTA
//            counts the destinations of its range;
//   barrier  (bounded spin)
//   phase 2  per-destination totals -> segment offsets (Sec. 4.2.2) and the
//            next active count (Sec. 4.2.3); each CTA's base per destination =
//            segment offset + the counts of the CTAs before it;
//   phase 3  each CTA re-reads its range of the out-queue and scatters it,
//            stably and grouped by destination, into the incoming queue;
//   barrier  then the next round, until no item is active.
//
// Step on arrival (policies with kFuseStep): phase 3 applies the next
// round's step to each item as it lands, so later rounds skip phase 1 and
// only count the destinations the scatter wrote; each item crosses HBM once
// per round.  When the next round is small enough (at most pushMax items)
// the scatter also adds each item's next destination into the count row of
// the CTA that will own the item's slot next round, so that round starts at
// phase 2: no count pass and one barrier instead of two.
//
// Because every step is per item and every scatter stable, queue order never
// depends on scheduling: round k's incoming queue equals the one of a serial
// round-by-round simulation.
//
// Every wait is bounded; a wait that gives up raises an abort flag that all
// CTAs check at the next barrier, and the kernel returns with a timeout status.
#pragma once

#include <functional>
#include <type_traits>
#include <utility>

#include "internal.cuh"
#include "rafi_device.cuh"

namespace rfi {

constexpr int kSyncGroups = 16;  // runs of consecutive CTAs whose destination counts are summed per round
// Independent runs one launch may carry (policies with kAppendRetired and
// steps on arrival): their items share the rank digits, each run has a
// retirement digit and a sink of its own.
constexpr int kMaxRuns = 4;
// a.result: {rounds, forwarded, status, retired}, then per run its rounds,
// then per run its retired count
constexpr int kResultWords = 4 + 2 * kMaxRuns;

// A destination word names a digit in its low 16 bits; the run an item
// belongs to rides in the high bits (0 for a launch of one run).  -1 (no
// destination) maps to digit 0xFFFF, above every valid digit.
__host__ __device__ __forceinline__ uint32_t digit_of(int32_t w) { return (uint32_t)w & 0xFFFFu; }
__host__ __device__ __forceinline__ uint32_t run_of(int32_t w) { return (uint32_t)w >> 16; }

struct GridSync {
    unsigned int count;    // arrivals at grid barriers so far
    unsigned int abort;    // set by a CTA whose wait gave up
    unsigned int work[2];  // work-phase chunk counters (round parity), dynamic policies
    unsigned int pad[28];
};

struct RoundsArgs {
    uint4 *in;
    uint4 *out;
    int32_t *dest;             // capacity rounded up to 4 entries + 4 (bulk-copied in 16-byte units)
    int32_t *dest2;            // the same size: second destination array (policies with kFuseStep)
    uint32_t *inOffset;        // numRanks + 1
    uint32_t *tot;             // 3 x gridDim.x rows of per-CTA destination counts (row stride: digits rounded to 4)
    uint32_t *grpTot;          // 3 x kSyncGroups rows (stride as tot): per-group destination totals
                               // (both tables: one set per iteration modulo 3, zero when the launch starts)
    GridSync *sync;
    unsigned long long *result;  // kResultWords: {rounds, forwarded, status, retired}, per-run rounds, per-run retired
    unsigned long long *numActiveOut;  // items still active when the kernel returns
    unsigned long long *roundLog;  // nullable: per round {t_start, t_work_end, t_barrier1, t_scatter_end, t_barrier2, n_in, n_next}
    uint4 *retiredOut;         // retirement sink (policies with kAppendRetired)
    unsigned long long retiredCap;
    unsigned long long *retiredCountOut;
    unsigned long long *seedCount;  // nullable: start from a seeded out-queue of this many items (kFuseStep)
    const uint4 *seedItems;         // nullable: the seeded items, read in place instead of from the out-queue
    long long spinLimit;       // bound of every grid-barrier wait, in SM clock cycles
    uint32_t missingArrivals;  // CTAs a grid barrier waits for beyond the grid (0; > 0 only to test timeouts)
    uint32_t pushMax;          // largest next round whose counts the scatter pushes (0: never; kFuseStep)
    uint32_t *smOf;            // gridDim.x words: each CTA's SM (rank skew)
    uint32_t skew;             // rank skew of large rounds' ranges, in 1/256 (0: equal ranges; <= 32)
    uint32_t maxRounds;
    uint32_t roundLogCap;
    uint32_t fuseStep;  // apply steps on arrival (policies with kFuseStep)
    int32_t numRanks;
    uint32_t numRuns;   // independent runs (1..kMaxRuns); retirement digit R + k is run k's
    uint32_t runCap;    // sink slots per run: run k retires into [k runCap, (k + 1) runCap)
    volatile unsigned long long *progress;  // nullable, host-mapped (policies with kProgress): the
                                            // retired items whose sink slots are final, after every round
};

constexpr int kRoundsBlock = 256;  // threads per CTA of a policy's default shape

// Policies that publish their retired count after every round (W::kProgress
// true) compile the store; the others carry no trace of it.
template <class W, class = void>
struct HasProgress : std::false_type {};
template <class W>
struct HasProgress<W, std::void_t<decltype(W::kProgress)>> : std::bool_constant<W::kProgress> {};

// A workload policy W (described at rounds_kernel) launched in another shape:
// K items per thread per tile, CTAS resident CTAs per SM to compile for,
// BLOCK threads per CTA.  Every shape computes the same rounds; the batched
// form's autotuner chooses among the shapes each policy compiles.
template <class W, int K, int CTAS, int BLOCK>
struct Shape : W {
    static constexpr int kItemsPerThread = K;
    static constexpr int kMinBlocksPerSM = CTAS;
    static constexpr int kBlock = BLOCK;
    Shape() = default;
    __host__ __device__ explicit Shape(const W &w) : W(w) {}
};

// What the host knows of a compiled shape.
struct ShapeInfo {
    int32_t block, itemsPerThread, ctasPerSM;
};

// Row stride (words) of the per-CTA count table: rows start 16-byte aligned
// so a run of rows can be staged with one bulk copy.
__host__ __device__ inline int rounds_row_stride(int R) { return (R + 3) / 4 * 4; }

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned int *p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void bulk_s2g(void *dstGlobal, const void *srcSmem, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dstGlobal),
                 "r"(smem_u32(srcSmem)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Orders this thread's generic-proxy global accesses with async-proxy
// (bulk copy) accesses to global memory, in either direction.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Lanes of the warp holding the same key (keys in [0, 2^nbits)): one ballot
// per key bit, the ballot form of __match_any_sync.
__device__ __forceinline__ unsigned peers_of(int key, int nbits)
{
    unsigned p = 0xFFFFFFFFu;
    for (int b = 0; b < nbits; ++b) {
        const bool bit = (key >> b) & 1;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, bit);
        p &= bit ? bal : ~bal;
    }
    return p;
}

__device__ __forceinline__ unsigned int atom_add_release(unsigned int *p, unsigned int v)
{
    unsigned int old;
    asm volatile("atom.release.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int *p, unsigned int v)
{
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Bounded grid barrier for a cooperative launch (all CTAs resident).
// The counter only grows (the launch zeroes it): barrier number `seq` (0, 1,
// ...) is complete once it reaches (G + missing) * (seq + 1), so nothing is
// ever reset.  Every CTA adds to the one counter and waits for the target
// (one atomic and one load on the critical path).  Arrivals are release
// operations and the waits acquire loads, which orders every CTA's writes
// before the barrier with every read after it.  `missing` is 0 in normal
// runs; a positive value names CTAs that never arrive, so every wait runs
// out after `limit` cycles (the timeout path, exercised without a fault).
// A wait that runs out raises the abort flag; every CTA that sees it while
// waiting gives up.  Returns false when this CTA gave up; the caller must
// then return.  A CTA that gave up arrives at no later barrier, so the others
// give up at their next one at the latest: a barrier that completes needs no
// extra read of the flag on its critical path.
__device__ inline bool barrier_wait_bounded(GridSync *gs, unsigned int target, long long limit)
{
    const long long t0 = clock64();
    for (unsigned int k = 0; ld_acquire(&gs->count) < target; ++k) {
        if ((k & 15u) == 15u) {
            if (ld_acquire(&gs->abort)) return false;
            if (clock64() - t0 > limit) {
                atomicExch(&gs->abort, 1u);
                return false;
            }
        }
        // (each poll is an L2 round trip; a 20 ns sleep between polls measured
        // 0.24 % slower over a joint launch of the three runs)
    }
    return true;
}

__device__ inline bool grid_barrier(GridSync *gs, unsigned int *sFlag, unsigned int seq, long long limit,
                                    unsigned int missing)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int target = (gridDim.x + missing) * (seq + 1u);
        const bool last = atom_add_release(&gs->count, 1u) + 1u == target;
        *sFlag = last ? 1u : (barrier_wait_bounded(gs, target, limit) ? 1u : 0u);
    }
    __syncthreads();
    return *sFlag != 0;
}

// The flat barrier in two halves, so a CTA can do work that needs no other
// CTA between arriving and waiting: grid_arrive (all threads; thread 0 adds
// to the counter, its earlier writes released) returns whether this CTA
// arrived last; grid_wait (all threads) waits for the rest, bounded, and
// returns false when this CTA gave up.
__device__ inline void grid_arrive(GridSync *gs, unsigned int seq, unsigned int *sLast, unsigned int missing)
{
    __syncthreads();
    if (threadIdx.x == 0)
        *sLast = atom_add_release(&gs->count, 1u) + 1u == (gridDim.x + missing) * (seq + 1u) ? 1u : 0u;
}

__device__ inline bool grid_wait(GridSync *gs, unsigned int *sFlag, unsigned int seq, const unsigned int *sLast,
                                 long long limit, unsigned int missing)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        *sFlag = *sLast ? 1u : (barrier_wait_bounded(gs, (gridDim.x + missing) * (seq + 1u), limit) ? 1u : 0u);
    }
    __syncthreads();
    return *sFlag != 0;
}

// Exclusive scan of v[0..n) in shared memory by a block of kB threads (n <= 8 kB).
template <int kB>
__device__ inline uint32_t rounds_block_scan(uint32_t *v, int n, uint32_t *tmp)
{
    constexpr int kWarps = kB / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __syncthreads();
    if (n <= 256) {
        // up to 256 entries: warp 0 alone, eight per lane, between two barriers
        if (warp == 0) {
            uint32_t x[8], sum = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int i = lane * 8 + j;
                const uint32_t t = i < n ? v[i] : 0u;
                x[j] = sum;
                sum += t;
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += t;
            }
            const uint32_t base = incl - sum;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int i = lane * 8 + j;
                if (i < n) v[i] = base + x[j];
            }
            if (lane == 31) tmp[kWarps] = incl;
        }
        __syncthreads();
        return tmp[kWarps];  // the next scan starts with a barrier before it writes tmp
    }
    uint32_t x[8], sum = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int i = tid * 8 + j;
        const uint32_t t = i < n ? v[i] : 0u;
        x[j] = sum;
        sum += t;
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < kWarps ? tmp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kWarps) tmp[lane] = wi - w;
        if (lane == 31) tmp[kWarps] = wi;
    }
    __syncthreads();
    const uint32_t base = tmp[warp] + incl - sum;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int i = tid * 8 + j;
        if (i < n) v[i] = base + x[j];
    }
    const uint32_t total = tmp[kWarps];
    __syncthreads();
    return total;
}

// Item j of a staged tile is V contiguous 16-byte vectors.  When a warp
// reads vector q of 32 consecutive items, each quarter warp (8 threads, one
// shared-memory wavefront) lands on the same few bank groups: 4-way conflicts
// for 64-byte items.  Each thread instead walks its item's vectors starting
// at a per-thread offset (position q xor r, r = (j V / 8) mod V), which puts
// the 8 threads of a quarter warp on 8 distinct 16-byte bank groups, and
// permutes the registers back with selects.  V a power of two up to 8; other
// V keep the plain order.
template <int V>
__device__ __forceinline__ uint32_t tile_rot(uint32_t j)
{
    if constexpr (V == 2 || V == 4 || V == 8) return (j * (uint32_t)V / 8u) & (uint32_t)(V - 1);
    else return 0u;
}

// t[q] <- t[q xor r] for all q (the xor permutation, one swap stage per bit of r)
template <int V>
__device__ __forceinline__ void xor_permute(uint4 (&t)[V], uint32_t r)
{
    if constexpr (V == 2 || V == 4 || V == 8) {
#pragma unroll
        for (int b = 1; b < V; b <<= 1) {
            const bool f = (r & (uint32_t)b) != 0u;
#pragma unroll
            for (int q = 0; q < V; ++q) {
                if (q & b) continue;
                const uint4 x = t[q], y = t[q | b];
                t[q] = f ? y : x;
                t[q | b] = f ? x : y;
            }
        }
    }
}

template <int V>
__device__ __forceinline__ void load_item_rot(const uint4 *s, uint32_t j, uint4 (&w)[V])
{
    const uint32_t r = tile_rot<V>(j);
#pragma unroll
    for (int q = 0; q < V; ++q) w[q] = s[j * V + ((uint32_t)q ^ r)];
    xor_permute<V>(w, r);
}

template <int V>
__device__ __forceinline__ void store_item_rot(uint4 *s, uint32_t j, const uint4 (&w)[V])
{
    const uint32_t r = tile_rot<V>(j);
    uint4 t[V];
#pragma unroll
    for (int q = 0; q < V; ++q) t[q] = w[q];
    xor_permute<V>(t, r);
#pragma unroll
    for (int q = 0; q < V; ++q) s[j * V + ((uint32_t)q ^ r)] = t[q];
}

// The vectors of an item a policy's step reads (W::kStepReadMask) and writes
// (W::kStepWriteMask).  A step that touches the whole item walks it in the
// rotated order; a partial one loads and stores only its own vectors (the
// rest of w is left zero and never written back).
template <class W>
__device__ __forceinline__ void load_step(const uint4 *s, uint32_t j, uint4 (&w)[W::V])
{
    constexpr unsigned kAll = (1u << W::V) - 1u;
    if constexpr ((W::kStepReadMask & kAll) == kAll) {
        load_item_rot<W::V>(s, j, w);
    } else {
#pragma unroll
        for (int q = 0; q < W::V; ++q)
            w[q] = ((W::kStepReadMask >> q) & 1u) ? s[j * W::V + q] : make_uint4(0u, 0u, 0u, 0u);
    }
}

template <class W>
__device__ __forceinline__ void store_step(uint4 *s, uint32_t j, const uint4 (&w)[W::V])
{
    constexpr unsigned kAll = (1u << W::V) - 1u;
    if constexpr ((W::kStepWriteMask & kAll) == kAll) {
        store_item_rot<W::V>(s, j, w);
    } else {
#pragma unroll
        for (int q = 0; q < W::V; ++q)
            if ((W::kStepWriteMask >> q) & 1u) s[j * W::V + q] = w[q];
    }
}

struct RoundsLayout {
    uint32_t items, dests, wc, cnt, start, base, tot, off, slotSrc, slotDst, tmp, flag, bar, ret, work, total;
};

__host__ __device__ inline uint32_t rounds_align(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }
inline size_t rounds_align_sz(size_t x, size_t a) { return (x + a - 1) / a * a; }

// items: two tile buffers (double buffering); the same bytes stage the
// per-CTA count rows in phase 2.  dests: the tiles' destinations.  D =
// destination digits (ranks, plus one retirement digit when the policy
// appends retired items).
__host__ __device__ inline RoundsLayout rounds_layout(uint32_t itemBytes, int D, uint32_t workBytes, uint32_t tile,
                                                  uint32_t warps)
{
    RoundsLayout L;
    uint32_t o = 0;
    L.items = o;   o = rounds_align(o + 2u * tile * itemBytes, 128);
    L.dests = o;   o = rounds_align(o + 2u * (tile + 4u) * 4u, 16);
    L.wc = o;      o = rounds_align(o + warps * D * 4u, 16);
    L.cnt = o;     o = rounds_align(o + D * 4u, 16);
    // The CTA's range counts (tot) live from a round's start until its count
    // row is written out, a tile's counts (cnt) from the scatter's first
    // ranking until the round ends: one array holds both.
    L.tot = L.cnt;
    L.start = o;   o = rounds_align(o + D * 4u, 16);
    L.base = o;    o = rounds_align(o + D * 4u, 16);
    L.off = o;     o = rounds_align(o + (D + 1) * 4u, 16);
    L.slotSrc = o; o = rounds_align(o + tile * 2u, 16);
    L.slotDst = o; o = rounds_align(o + tile * 4u, 16);
    L.tmp = o;     o = rounds_align(o + (warps + 1) * 4u, 16);
    L.flag = o;    o = rounds_align(o + 4u, 16);
    L.bar = o;     o = rounds_align(o + 16u, 16);
    L.ret = o;     o = rounds_align(o + kMaxRuns * 4u, 16);
    L.work = o;    o = rounds_align(o + workBytes, 16);
    L.total = o;
    return L;
}

// The workload policy W provides:
//   static constexpr int V;               16-byte vectors per item
//   static constexpr bool kAppendRetired; retired items go, stably, to the
//                                         retirement sink (else: retire())
//   static constexpr bool kDynamicWork;   long per-item work: a work phase of its
//                                         own over the whole queue, before the scatter
//   static constexpr bool kGridStride;    (kDynamicWork) items by grid stride rather
//                                         than dynamically handed-out chunks
//   static constexpr int kMinBlocksPerSM; resident CTAs per SM to compile for
//   static constexpr int kItemsPerThread; tile = kBlock x this many items
//   static constexpr int kBlock;          threads per CTA (multiple of 32)
//   static constexpr bool kFuseStep;      short, even per-item work: the scatter
//                                         applies the next round's step on arrival
//   uint32_t smemBytes() const;           its own shared memory
//   void load_smem(void *s) const;        fill it (all threads; a barrier follows)
//   int32_t step(uint4 (&w)[V], int32_t rank, uint32_t round, const void *s) const;
//       advances one item: returns the destination rank (w updated) or -1 to retire;
//       in a launch of several runs `rank` is the item's destination word (run in
//       the high bits, see digit_of) and the returned rank carries the same run
//   void retire(const uint4 (&w)[V]) const;  (used when !kAppendRetired)
template <class W>
__global__ void __launch_bounds__(W::kBlock, W::kMinBlocksPerSM) rounds_kernel(RoundsArgs a, W work)
{
    constexpr int V = W::V;
    constexpr int kB = W::kBlock;  // threads per CTA
    constexpr int kWarps = kB / 32;
    constexpr uint32_t kItemBytes = 16u * V;
    constexpr int kK = W::kItemsPerThread;  // items per thread per tile
    constexpr uint32_t kTile = kB * kK;
    constexpr uint32_t kTileVecs = kTile * V;
    constexpr uint32_t kRetFlag = 0x80000000u;
    constexpr bool kFuse = W::kFuseStep && !W::kDynamicWork;
    static_assert((W::kStepReadMask & ((1u << V) - 1u)) != 0u, "a step reads part of its item");
    extern __shared__ __align__(128) unsigned char smem[];
    const int R = a.numRanks;
    const int K = W::kAppendRetired ? (int)a.numRuns : 1;  // independent runs in the launch
    const int D = R + (W::kAppendRetired ? K : 0);  // digits: ranks (+ one retirement digit per run)
    const int Dp = rounds_row_stride(D);
    const RoundsLayout L = rounds_layout(kItemBytes, D, work.smemBytes(), kTile, kWarps);
    uint4 *sBuf = reinterpret_cast<uint4 *>(smem + L.items);  // two tiles of kTileVecs
    uint32_t *sRows = reinterpret_cast<uint32_t *>(smem + L.items) + kTileVecs * 4u;  // tile buffer 1
    int32_t *sDst = reinterpret_cast<int32_t *>(smem + L.dests);  // two tiles of kTile + 4
    uint32_t *wc = reinterpret_cast<uint32_t *>(smem + L.wc);
    uint32_t *dCnt = reinterpret_cast<uint32_t *>(smem + L.cnt);
    uint32_t *dStart = reinterpret_cast<uint32_t *>(smem + L.start);
    uint32_t *dBase = reinterpret_cast<uint32_t *>(smem + L.base);
    uint32_t *sTot = reinterpret_cast<uint32_t *>(smem + L.tot);
    uint32_t *sOff = reinterpret_cast<uint32_t *>(smem + L.off);
    uint16_t *slotSrc = reinterpret_cast<uint16_t *>(smem + L.slotSrc);
    uint32_t *slotDst = reinterpret_cast<uint32_t *>(smem + L.slotDst);
    uint32_t *tmp = reinterpret_cast<uint32_t *>(smem + L.tmp);
    unsigned int *sFlag = reinterpret_cast<unsigned int *>(smem + L.flag);
    uint32_t *sRet = reinterpret_cast<uint32_t *>(smem + L.ret);  // per run: items retired so far
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);  // bar[0], bar[1]: one per tile buffer
    void *sWork = smem + L.work;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, c = blockIdx.x;
    const int nbits = 32 - __clz(D);  // keys 0..D (D = no item)
    const uint32_t rowsPerStage = (kTileVecs * 16u) / (uint32_t)(Dp * 4);
    // prefix groups: kSyncGroups runs of consecutive CTAs
    const int grpSize = (G + kSyncGroups - 1) / kSyncGroups;
    const int grp = c / grpSize, grpStart = grp * grpSize;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async_smem();
    }
    if (tid < kMaxRuns) sRet[tid] = 0u;
    work.load_smem(sWork);
    __syncthreads();

    uint32_t par0 = 0u, par1 = 0u;     // phase parity of bar[0], bar[1]
    bool pend0 = false, pend1 = false;  // thread 0: a bulk load into the buffer is in flight
    // issue bulk loads of `bytes` at src (and optionally `bytes2` at src2) into buffer `buf` (thread 0)
    auto issue_bytes = [&](int buf, void *dst, const void *src, uint32_t bytes, void *dst2, const void *src2,
                           uint32_t bytes2) {
        fence_proxy_async_smem();
        fence_proxy_async_global();
        mbar_arrive_expect_tx(&bar[buf], bytes + bytes2);
        bulk_g2s(dst, src, bytes, &bar[buf]);
        if (bytes2) bulk_g2s(dst2, src2, bytes2, &bar[buf]);
        if (buf) pend1 = true;
        else pend0 = true;
    };
    // wait for buffer `buf` (all threads).  On a timeout: raise the abort flag,
    // let every copy still in flight land (bounded), return false.
    auto wait = [&](int buf) -> bool {
        bool ok;
        if (buf) {
            ok = mbar_wait_bounded(&bar[1], par1);
            par1 ^= 1u;
            pend1 = false;
        } else {
            ok = mbar_wait_bounded(&bar[0], par0);
            par0 ^= 1u;
            pend0 = false;
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(&a.sync->abort, 1u);
                (void)mbar_wait_bounded(&bar[buf], (buf ? par1 : par0) ^ 1u);
                if (buf == 0 && pend1) (void)mbar_wait_bounded(&bar[1], par1);
                if (buf == 1 && pend0) (void)mbar_wait_bounded(&bar[0], par0);
            }
            return false;
        }
        return true;
    };
    // CTA cc's range of a round with m items over g CTAs: boundaries rounded up
    // to 16 items (so a small round lands on the first CTAs)
    auto bound = [&](uint32_t m, int cc, int g) -> uint32_t {
        const unsigned long long v = (((unsigned long long)m * cc) / g + 15ull) & ~15ull;
        return (uint32_t)(v < m ? v : m);
    };
    // Once a round fits in one tile, CTA 0 finishes the run alone: the other
    // CTAs return and the round barriers become block barriers.  (Rounds of two
    // to four tiles measured 10-17 us on one CTA against about 10 us on the grid.)
    constexpr uint32_t kSoloItems = kTile;
    constexpr uint32_t kSkewItems = 1u << 19;
    constexpr int kCountLoads = 4;  // 16-byte destination loads in flight per thread in the count pass
    bool solo = false;
    unsigned int barrierSeq = 0;  // grid barriers passed (every CTA passes the same ones)
    auto round_barrier = [&]() -> bool {
        if (!solo) return grid_barrier(a.sync, sFlag, barrierSeq++, a.spinLimit, a.missingArrivals);
        __threadfence();
        __syncthreads();
        return true;
    };

    // A seeded start (kFuseStep policies): the out-queue P0 holds the seeded
    // items with their first ranks as destinations; a pre-round delivers them
    // (not counted as a round, its deliveries not as forwards), applying
    // round 0's step on arrival.
    bool pre = kFuse && a.fuseStep && a.seedCount != nullptr;
    uint32_t n = pre ? (uint32_t)*a.seedCount : a.inOffset[R];
    unsigned long long forwarded = 0, retiredSoFar = 0;
    uint32_t round = 0, it = 0;  // it: iterations including the pre-round (parity of the round counters)
    bool failed = false;
    // Step on arrival (policies with kFuseStep): the scatter of round k applies
    // round k+1's step to each item as it lands in its destination's segment,
    // so the next round starts from stepped items and only counts their
    // destinations.  Stepped items live in one of two (items, destinations)
    // pairs, P0 = (out, dest) and P1 = (in, dest2); xsel names the current one.
    // `fresh`: the incoming queue holds unstepped items (round 0, or after a
    // plain scatter), which phase 1 steps into P0.
    bool fresh = !pre;
    // `pushed`: the previous scatter already added this round's destinations
    // into the count rows, so the round starts at phase 2.
    bool pushed = false;
    uint32_t xsel = 0u;
    auto curItemsOf = [&](uint32_t x) { return x ? a.in : a.out; };
    auto curDestOf = [&](uint32_t x) { return x ? a.dest2 : a.dest; };

    // Ranks a staged tile (items sItems, destinations dts, cnt entries)
    // stably by destination digit, applying round qs's step to every item
    // bound for a rank when doFuse (its new destination replaces the staged
    // one); fills dCnt, dStart (the tile's slots grouped by digit) and
    // slotSrc / slotDst (position = dBase[d] + rank within d; the retirement
    // flag for the retirement digits R + k).  With ownBases the tile is a whole
    // round on its own: dBase[d] = dStart[d] for ranks, and for run k's
    // retirement digit its sink base k runCap plus its retired count so far.
    // Returns the number of valid items.  All threads; ends with a barrier.
    // carryPrev: first add the previous tile's counts (still in dCnt) to dBase.
    // First half (needs no other CTA): per-warp ranks (myD, myR, wc) and the
    // fused step; second half: per-tile counts, slots and positions.
    auto rank_a = [&](uint4 *sItems, int32_t *dts, uint32_t cnt, bool doFuse, uint32_t qs, int (&myD)[kK],
                      uint32_t (&myR)[kK]) {
#pragma unroll
        for (int k = 0; k < kK; ++k) {
            const uint32_t idx = (uint32_t)(warp * 32 * kK + k * 32 + lane);
            const int32_t dw = idx < cnt ? dts[idx] : -1;  // destination word (digit and run)
            const int32_t d = (int32_t)digit_of(dw);
            const bool valid = (uint32_t)d < (uint32_t)D;
            const int key = valid ? d : D;
            const unsigned peers = peers_of(key, nbits);
            const int leader = __ffs(peers) - 1;
            uint32_t old = 0;
            if (valid && lane == leader) {
                old = wc[warp * D + d];
                wc[warp * D + d] = old + (uint32_t)__popc(peers);
            }
            old = __shfl_sync(0xFFFFFFFFu, old, leader);
            __syncwarp();
            myD[k] = valid ? d : -1;
            myR[k] = old + (uint32_t)__popc(peers & lanemask_lt());
            if (doFuse && valid && d < R) {
                uint4 w[V];
                if constexpr (W::kAppendRetired) load_step<W>(sItems, idx, w);
                else load_item_rot<V>(sItems, idx, w);  // retire() takes the whole item
                int32_t d2 = work.step(w, dw, qs, sWork);
                if (d2 >= 0) {
                    store_step<W>(sItems, idx, w);
                } else if (W::kAppendRetired) {
                    d2 = R + (int32_t)run_of(dw);  // the run's retirement digit
                } else {
                    work.retire(w);
                }
                dts[idx] = d2;
            }
        }
        if (doFuse) fence_proxy_async_smem();  // generic writes before the buffer's next bulk load
        __syncthreads();
    };
    auto rank_b = [&](bool ownBases, bool carryPrev, const int (&myD)[kK], const uint32_t (&myR)[kK]) -> uint32_t {
        for (int e = tid; e < D; e += kB) {
            uint32_t sum = 0;
#pragma unroll
            for (int ww = 0; ww < kWarps; ++ww) {
                const uint32_t v = wc[ww * D + e];
                wc[ww * D + e] = sum;
                sum += v;
            }
            if (carryPrev) dBase[e] += dCnt[e];
            dCnt[e] = sum;
            dStart[e] = sum;
        }
        const uint32_t nValid = rounds_block_scan<kB>(dStart, D, tmp);
        if (ownBases) {
            for (int e = tid; e < D; e += kB)
                dBase[e] = (W::kAppendRetired && e >= R) ? (uint32_t)(e - R) * a.runCap + sRet[e - R] : dStart[e];
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < kK; ++k) {
            if (myD[k] >= 0) {
                const int d = myD[k];
                const uint32_t within = wc[warp * D + d] + myR[k];
                const uint32_t slot = dStart[d] + within;
                slotSrc[slot] = (uint16_t)(warp * 32 * kK + k * 32 + lane);
                slotDst[slot] = (dBase[d] + within) | (W::kAppendRetired && d >= R ? kRetFlag : 0u);
            }
        }
        __syncthreads();
        return nValid;
    };
    auto rank_tile = [&](uint4 *sItems, int32_t *dts, uint32_t cnt, bool doFuse, uint32_t qs, bool ownBases,
                         bool carryPrev) -> uint32_t {
        int myD[kK];
        uint32_t myR[kK];
        rank_a(sItems, dts, cnt, doFuse, qs, myD, myR);
        return rank_b(ownBases, carryPrev, myD, myR);
    };

    // Co-resident CTAs do not get equal shares of their SM's memory
    // bandwidth: the older ones (lower blockIdx among the CTAs on an SM) are
    // served first and finish equal ranges early, and the SM idles on its
    // last CTA.  With a.skew > 0, rounds of at least kSkewItems items give
    // CTA c a range in proportion to w = 256 + skew (k - 1 - 2 rho), rho its
    // launch order among the k CTAs on its SM: [W0, W1) of the grid's Wt.
    // The weights come from every CTA's %smid, exchanged once per launch.
    unsigned long long W0 = 0, W1 = 0, Wt = 0;
    bool skewed = a.skew > 0u && G > 1;
    if (skewed) {
        if (tid == 0) {
            unsigned sm;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
            a.smOf[c] = sm;
        }
        if (!grid_barrier(a.sync, sFlag, barrierSeq++, a.spinLimit, a.missingArrivals)) {
            failed = true;
        } else {
            // every CTA's SM in the tile buffer (unused until round 0 stages a tile)
            uint32_t *sSm = reinterpret_cast<uint32_t *>(sBuf);
            uint32_t *acc = sSm + G;
            for (int e = tid; e < G; e += kB) sSm[e] = __ldcg(a.smOf + e);
            if (tid < 3) acc[tid] = 0u;
            __syncthreads();
            uint32_t below = 0, all = 0, mine = 0;
            for (int e = tid; e < G; e += kB) {
                int rho = 0, k = 0;
                for (int f = 0; f < G; ++f) {
                    const bool same = sSm[f] == sSm[e];
                    k += same;
                    rho += same && f < e;
                }
                const uint32_t w = (uint32_t)max(1, 256 + (int)a.skew * (k - 1 - 2 * rho));
                all += w;
                if (e < c) below += w;
                if (e == c) mine = w;
            }
            atomicAdd(&acc[0], below);
            atomicAdd(&acc[1], mine);
            atomicAdd(&acc[2], all);
            __syncthreads();
            W0 = acc[0];
            W1 = W0 + acc[1];
            Wt = acc[2];
            __syncthreads();  // the tile buffer is free again
        }
    }
    // CTA c's range under the skew: boundaries rounded up to 16 items
    auto wbound = [&](uint32_t m, unsigned long long W) -> uint32_t {
        const unsigned long long v = ((unsigned long long)m * W / Wt + 15ull) & ~15ull;
        return (uint32_t)(v < m ? v : m);
    };

    for (;; ++it) {
        if (failed || n == 0 || (!pre && round >= a.maxRounds)) break;
        if (!solo && n <= kSoloItems) {
            solo = true;
            if (c != 0) break;
        }
        if (kFuse && a.fuseStep && solo && !fresh && !pre && n <= kTile && round + 2u < a.maxRounds) {
            // ---- on-chip tail: CTA 0 alone with the whole queue in shared memory.
            // Each round ranks the stepped queue (tile A), applies the next
            // round's step on arrival and writes the next queue into tile B;
            // retired items go to the sink.  Two rounds before maxRounds the
            // queue is handed back to P0 for the general path's plain last round.
            if (tid == 0)
                issue_bytes(0, sBuf, curItemsOf(xsel), n * kItemBytes, sDst, curDestOf(xsel), ((n + 3u) & ~3u) * 4u);
            if (!wait(0)) {
                failed = true;
                break;
            }
            uint32_t A = 0;
            while (n > 0 && round + 2u < a.maxRounds) {
                const bool lr = a.roundLog && tid == 0 && round < a.roundLogCap;
                if (lr) a.roundLog[7 * round + 0] = globaltimer();
                for (int e = lane; e < D; e += 32) wc[warp * D + e] = 0u;
                __syncwarp();
                uint4 *iA = sBuf + A * kTileVecs, *iB = sBuf + (A ^ 1u) * kTileVecs;
                int32_t *dA = sDst + A * (kTile + 4u), *dB = sDst + (A ^ 1u) * (kTile + 4u);
                const uint32_t nValid = rank_tile(iA, dA, n, true, round + 1u, true, false);
                const uint32_t nNext = W::kAppendRetired ? dStart[R] : nValid;
                uint32_t retiredNow = 0u;
                if (W::kAppendRetired) {
                    for (int k = 0; k < K; ++k) retiredNow += dCnt[R + k];
                    // (sRet is next read by the following round's ranking, after barriers)
                    if (tid < K && dCnt[R + tid]) {
                        sRet[tid] += dCnt[R + tid];
                        if (c == 0) a.result[4 + tid] = round + 1u;  // the run's last round so far
                    }
                }
                if (lr) a.roundLog[7 * round + 1] = a.roundLog[7 * round + 2] = globaltimer();
                for (uint32_t slot = tid; slot < nValid; slot += kB) {
                    const uint32_t dst = slotDst[slot];
                    const uint32_t src = slotSrc[slot];
                    const uint32_t rot = tile_rot<V>(src);
                    const bool ret = W::kAppendRetired && (dst & kRetFlag);
                    const uint32_t pos = dst & ~kRetFlag;
                    uint4 *to = ret ? (pos < a.retiredCap ? a.retiredOut + (size_t)pos * V : nullptr) : iB + pos * V;
                    if (to) {
#pragma unroll
                        for (int qq = 0; qq < V; ++qq) {
                            const uint32_t p = (uint32_t)qq ^ rot;
                            to[p] = iA[src * V + p];
                        }
                    }
                    if (!ret) dB[pos] = dA[src];
                }
                __syncthreads();
                if (lr) {
                    a.roundLog[7 * round + 3] = a.roundLog[7 * round + 4] = globaltimer();
                    a.roundLog[7 * round + 5] = n;
                    a.roundLog[7 * round + 6] = nNext;
                }
                retiredSoFar += retiredNow;
                if constexpr (HasProgress<W>::value) {
                    if (a.progress && tid == 0) {
                        __threadfence_system();
                        *a.progress = retiredSoFar;
                    }
                }
                forwarded += nNext;
                n = nNext;
                A ^= 1u;
                ++round;
            }
            if (n > 0) {
                // hand the stepped queue back in P0 and clear the round counters
                uint4 *iA = sBuf + A * kTileVecs;
                const int32_t *dA = sDst + A * (kTile + 4u);
                for (uint32_t v = tid; v < n * V; v += kB) a.out[v] = iA[v];
                for (uint32_t i = tid; i < n; i += kB) a.dest[i] = dA[i];
                for (int e = tid; e < 3 * kSyncGroups * Dp; e += kB) a.grpTot[e] = 0u;
                xsel = 0u;
            } else {
                for (int e = tid; e <= R; e += kB) a.inOffset[e] = 0u;
            }
            fence_proxy_async_global();
            __threadfence();
            __syncthreads();
            continue;
        }
        const int g = solo ? 1 : G;
        // count tables of this iteration: set it mod 3 (the previous scatter may
        // push into it; phase 2 clears the set two iterations ahead)
        const uint32_t b3 = it % 3u;
        const bool logRound = !pre && a.roundLog && c == 0 && tid == 0 && round < a.roundLogCap;
        if (logRound) a.roundLog[7 * round + 0] = globaltimer();
        // segment offsets: phase 1 ranks its items by them (a stepped queue needs none)
        if (fresh || W::kDynamicWork)
            for (int e = tid; e <= R; e += kB) sOff[e] = a.inOffset[e];
        for (int e = tid; e < D; e += kB) sTot[e] = 0u;
        __syncthreads();
        // (a round whose counts were pushed keeps the equal ranges the push assumed)
        const bool weighted = skewed && !solo && !pushed && n >= kSkewItems;
        const uint32_t lo = weighted ? wbound(n, W0) : bound(n, c, g);
        const uint32_t hi = weighted ? wbound(n, W1) : bound(n, c + 1, g);
        const uint32_t nt = (hi - lo + kTile - 1) / kTile;

        // ---- phase 1: work step, write back to the same slots ------------------
        // Policies with long, uneven per-item work (W::kDynamicWork) take
        // 32-item chunks from a round counter instead of a fixed range; each
        // CTA then counts its own range's destinations after the barrier.
        const bool dynamic = W::kDynamicWork && !solo;
        // A run that stops at maxRounds must leave an unstepped queue in `in`:
        // the last round scatters plainly, from P0, so the round before it
        // fuses only when that lands its items in P0.
        const uint32_t q = pre ? 0u : round + 1u;  // the round whose step the scatter may apply
        const bool fuse = kFuse && a.fuseStep && q < a.maxRounds && !(q + 1u == a.maxRounds && xsel == 0u);
        // the pre-round may read the seeded items where the caller keeps them
        const uint4 *const curItems = (pre && a.seedItems) ? a.seedItems : curItemsOf(xsel);
        int32_t *const curDest = curDestOf(xsel);
        uint4 *const nxtItems = fuse ? (xsel ? a.out : a.in) : a.in;
        int32_t *const nxtDest = xsel ? a.dest : a.dest2;
        // stage tile t of this CTA's range (items and destinations) into buffer buf
        auto issue3 = [&](int buf, uint32_t bb) {
            const uint32_t cc = min(kTile, hi - bb);
            issue_bytes(buf, sBuf + buf * kTileVecs, curItems + (size_t)bb * V, cc * kItemBytes,
                        sDst + buf * (kTile + 4u), curDest + bb, ((cc + 3u) & ~3u) * 4u);
        };
        // A stepped queue is final when the round starts: its first tile is
        // staged now, so the copy overlaps the count pass and the barrier.
        const bool prefetched = !fresh && !dynamic && nt > 0;
        if (prefetched && tid == 0) issue3(0, lo);
        if (dynamic) {
            // W::kGridStride: thread t of the grid takes items t, t + 256 G, ...
            // (no atomics; for steps of similar cost).  Otherwise each warp
            // takes 32-item chunks from the round's counter.
            unsigned int *ticket = &a.sync->work[it & 1u];
            uint32_t strided = (uint32_t)c * kB + (uint32_t)warp * 32u;
            for (;;) {
                uint32_t base = 0;
                if (W::kGridStride) {
                    base = strided;
                    strided += (uint32_t)G * kB;
                } else {
                    if (lane == 0) base = atomicAdd(ticket, 32u);
                    base = __shfl_sync(0xFFFFFFFFu, base, 0);
                }
                if (base >= n) break;
                const uint32_t i = base + lane;
                if (i < n) {
                    uint4 w[V];
#pragma unroll
                    for (int q = 0; q < V; ++q) w[q] = __ldcg(a.in + (size_t)i * V + q);
                    int32_t d = work.step(w, rf::rankOf(sOff, R, i), round, sWork);
                    if (d >= 0) {
#pragma unroll
                        for (int q = 0; q < V; ++q) a.out[(size_t)i * V + q] = w[q];
                    } else if (W::kAppendRetired) {
#pragma unroll
                        for (int q = 0; q < V; ++q) a.out[(size_t)i * V + q] = w[q];
                        d = R;
                    } else {
                        work.retire(w);
                    }
                    a.dest[i] = d;
                }
            }
            if (c == 0 && tid == 0) a.sync->work[(it + 1u) & 1u] = 0u;  // next round's counter
        }
        if (!dynamic && fresh && tid == 0 && nt) {
            const uint32_t cnt0 = min(kTile, hi - lo);
            issue_bytes(0, sBuf, a.in + (size_t)lo * V, cnt0 * kItemBytes, nullptr, nullptr, 0u);
        }
        for (uint32_t t = 0; !dynamic && fresh && t < nt; ++t) {
            const int buf = t & 1;
            const uint32_t b = lo + t * kTile;
            const uint32_t cnt = min(kTile, hi - b);
            if (tid == 0 && t + 1 < nt) {
                bulk_wait_read();  // the store of tile t-1 has left buffer buf^1
                const uint32_t nb = b + kTile;
                issue_bytes(buf ^ 1, sBuf + (buf ^ 1) * kTileVecs, a.in + (size_t)nb * V,
                            min(kTile, hi - nb) * kItemBytes, nullptr, nullptr, 0u);
            }
            if (!wait(buf)) {
                failed = true;
                break;
            }
            uint4 *sItems = sBuf + buf * kTileVecs;
#pragma unroll
            for (int k = 0; k < kK; ++k) {
                const uint32_t j = (uint32_t)(k * kB + tid);
                const bool valid = j < cnt;
                int32_t d = -1;
                if (valid) {
                    uint4 w[V];
                    if constexpr (W::kAppendRetired) load_step<W>(sItems, j, w);
                    else load_item_rot<V>(sItems, j, w);  // retire() takes the whole item
                    const int32_t rank = rf::rankOf(sOff, R, b + j);
                    d = work.step(w, rank, round, sWork);
                    if (d >= 0) {
                        store_step<W>(sItems, j, w);
                    } else if (W::kAppendRetired) {
                        d = R;  // the retirement digit: scattered to the sink in phase 3
                    } else {
                        work.retire(w);
                    }
                    a.dest[b + j] = d;
                }
                const int key = (valid && d >= 0) ? d : D;
                const unsigned peers = peers_of(key, nbits);
                if (key < D && lane == __ffs(peers) - 1) atomicAdd(&sTot[key], (uint32_t)__popc(peers));
            }
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) bulk_s2g(a.out + (size_t)b * V, sItems, cnt * kItemBytes);
        }
        if (tid == 0) bulk_wait_all();
        if (logRound && fresh) a.roundLog[7 * round + 1] = globaltimer();
        if (dynamic) {
            fence_proxy_async_global();
            if (!round_barrier()) {
                failed = true;
                break;
            }
        }
        if (dynamic || (!fresh && !pushed)) {
            // count the destinations of this CTA's range into per-warp rows:
            // 16-byte loads (lo is a multiple of 16 items), kCountLoads in
            // flight per thread; the padded array covers the last vector's tail
            for (int e = lane; e < D; e += 32) wc[warp * D + e] = 0u;
            __syncwarp();
            const int4 *dv = reinterpret_cast<const int4 *>(curDest + lo);
            const uint32_t nv = (hi - lo + 3u) / 4u;
            for (uint32_t v0 = 0; v0 < nv; v0 += (uint32_t)kCountLoads * kB) {
                int4 x[kCountLoads];
#pragma unroll
                for (int u = 0; u < kCountLoads; ++u) {
                    const uint32_t v = v0 + (uint32_t)u * kB + tid;
                    x[u] = v < nv ? __ldcg(dv + v) : make_int4(-1, -1, -1, -1);
                }
#pragma unroll
                for (int u = 0; u < kCountLoads; ++u) {
                    const uint32_t i = lo + 4u * (v0 + (uint32_t)u * kB + tid);
                    const int32_t e4[4] = {x[u].x, x[u].y, x[u].z, x[u].w};
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const uint32_t dg = digit_of(e4[m]);
                        if (i + m < hi && dg < (uint32_t)D) atomicAdd(&wc[warp * D + dg], 1u);
                    }
                }
            }
            __syncthreads();
            for (int e = tid; e < D; e += kB) {
                uint32_t sum = 0;
#pragma unroll
                for (int ww = 0; ww < kWarps; ++ww) sum += wc[ww * D + e];
                sTot[e] += sum;
            }
            __syncthreads();
            if (logRound && !fresh) a.roundLog[7 * round + 1] = globaltimer();
        }
        if (!failed && !pushed) {
            for (int e = tid; e < D; e += kB) {
                const uint32_t v = sTot[e];
                a.tot[((size_t)b3 * G + c) * Dp + e] = v;
                if (v) atomicAdd(&a.grpTot[(b3 * kSyncGroups + grp) * Dp + e], v);
            }
        }
        fence_proxy_async_global();
        if (failed) break;
        // With the first tile staged early, its per-warp ranks and fused step
        // (the half that needs no other CTA) run between arriving at the
        // first barrier and waiting for it.
        int myD0[kK];
        uint32_t myR0[kK];
        bool earlyDone = false;
        if (pushed) {
            // every count row was complete when the previous round's last barrier passed
            if (logRound) a.roundLog[7 * round + 1] = globaltimer();
        } else if (!solo && prefetched) {
            grid_arrive(a.sync, barrierSeq, sFlag + 1, a.missingArrivals);
            for (int e = lane; e < D; e += 32) wc[warp * D + e] = 0u;
            __syncwarp();
            if (!wait(0)) {
                failed = true;
            } else {
                rank_a(sBuf, sDst, min(kTile, hi - lo), fuse, q, myD0, myR0);
                earlyDone = true;
            }
            const bool ok = grid_wait(a.sync, sFlag, barrierSeq++, sFlag + 1, a.spinLimit, a.missingArrivals);
            if (failed || !ok) {
                failed = true;
                break;
            }
        } else if (!round_barrier()) {
            failed = true;
            break;
        }
        if (logRound) a.roundLog[7 * round + 2] = globaltimer();

        // ---- phase 2: offsets, next count, this CTA's base per destination -----
        // One bulk copy stages every group's totals and the rows of the CTAs
        // before this one in its group: per destination, the total is the sum
        // of the group rows, and this CTA's base the sum of the group rows
        // before its group plus the member rows (in chunks when they do not
        // fit the buffer).
        {
            const uint32_t nGroups = (uint32_t)((G + grpSize - 1) / grpSize);
            const uint32_t mRows = (uint32_t)(c - grpStart);
            const uint32_t *gSrc = a.grpTot + (size_t)b3 * kSyncGroups * Dp;
            const uint32_t *mSrc = a.tot + ((size_t)b3 * G + grpStart) * Dp;
            for (int e = tid; e < D; e += kB) {
                dStart[e] = 0u;
                dBase[e] = 0u;
            }
            const uint32_t allRows = nGroups + mRows;
            for (uint32_t r0 = 0; r0 < allRows && !failed; r0 += rowsPerStage) {
                const uint32_t rows = min(rowsPerStage, allRows - r0);
                if (tid == 0) {
                    // rows r0 .. r0 + rows - 1 of [group rows, member rows]
                    const uint32_t g0 = r0 < nGroups ? min(rows, nGroups - r0) : 0u;
                    const uint32_t m0 = r0 < nGroups ? 0u : r0 - nGroups;
                    if (g0 == 0)
                        issue_bytes(1, sRows, mSrc + (size_t)m0 * Dp, rows * Dp * 4u, nullptr, nullptr, 0u);
                    else if (g0 == rows)
                        issue_bytes(1, sRows, gSrc + (size_t)r0 * Dp, rows * Dp * 4u, nullptr, nullptr, 0u);
                    else
                        issue_bytes(1, sRows, gSrc + (size_t)r0 * Dp, g0 * Dp * 4u, sRows + g0 * Dp, mSrc,
                                    (rows - g0) * Dp * 4u);
                }
                if (!wait(1)) {
                    failed = true;
                    break;
                }
                for (int e = tid; e < D; e += kB) {
                    uint32_t tot = 0, before = 0;
                    for (uint32_t rr = 0; rr < rows; ++rr) {
                        const uint32_t row = r0 + rr;
                        const uint32_t v = sRows[rr * Dp + e];
                        if (row < nGroups) {
                            tot += v;
                            if (row < (uint32_t)grp) before += v;
                        } else {
                            before += v;
                        }
                    }
                    dStart[e] += tot;
                    dBase[e] += before;
                }
                __syncthreads();
            }
        }
        uint32_t retiredNow = 0u;
        if (W::kAppendRetired)
            for (int k = 0; k < K; ++k) retiredNow += dStart[R + k];
        const uint32_t nNext = rounds_block_scan<kB>(dStart, R, tmp);  // ranks only
        if (W::kAppendRetired && tid < K) {
            // run tid's retirement digit: its sink base, then its running count
            const uint32_t rn = dStart[R + tid];
            dStart[R + tid] = (uint32_t)tid * a.runCap + sRet[tid];
            sRet[tid] += rn;
            if (c == 0 && rn) a.result[4 + tid] = round + 1u;  // the run's last round so far
        }
        __syncthreads();
        for (int e = tid; e < D; e += kB) dBase[e] += dStart[e];
        // clear the count tables of iteration it + 2 (last read in phase 2 of
        // iteration it - 1; first written after this round's last barrier)
        const uint32_t bz = (b3 + 2u) % 3u;
        for (int e = tid; e < D; e += kB) a.tot[((size_t)bz * G + c) * Dp + e] = 0u;
        if (c == 0) {
            for (int e = tid; e < R; e += kB) a.inOffset[e] = dStart[e];
            for (int e = tid; e < kSyncGroups * Dp; e += kB) a.grpTot[(size_t)bz * kSyncGroups * Dp + e] = 0u;
            if (tid == 0) a.inOffset[R] = nNext;
        }
        // Push the next round's counts from this scatter when that round is a
        // grid round of at most pushMax items: its owner of slot p is the last
        // CTA whose range starts at or before p's 16-item chunk.  Every CTA
        // takes the same decision (nNext is a grid-wide total).
        const bool push = kFuse && fuse && !solo && nNext > kSoloItems && nNext <= a.pushMax;
        uint32_t *const totNext = a.tot + (size_t)((b3 + 1u) % 3u) * G * Dp;
        uint32_t *const grpNext = a.grpTot + (size_t)((b3 + 1u) % 3u) * kSyncGroups * Dp;
        if (!pre) forwarded += nNext;
        retiredSoFar += retiredNow;
        __syncthreads();

        // ---- phase 3: stable scatter of this CTA's range -----------------------
        if (tid == 0 && nt && !failed && !prefetched) issue3(0, lo);
        for (uint32_t t = 0; t < nt && !failed; ++t) {
            const int buf = t & 1;
            const uint32_t b = lo + t * kTile;
            const uint32_t cnt = min(kTile, hi - b);
            int32_t *dts = sDst + buf * (kTile + 4u);
            uint4 *sItems = sBuf + buf * kTileVecs;
            uint32_t nValid;
            // The next tile goes into the other buffer once every thread is past
            // the scatter that last read it: after this tile's wait (a block
            // barrier), or at once for the first tile (phase 2 ended with one).
            if (t == 0 && earlyDone) {
                if (tid == 0 && t + 1 < nt) issue3(buf ^ 1, b + kTile);
                nValid = rank_b(false, false, myD0, myR0);
            } else {
                for (int e = lane; e < D; e += 32) wc[warp * D + e] = 0u;
                if (!wait(buf)) {
                    failed = true;
                    break;
                }
                if (tid == 0 && t + 1 < nt) issue3(buf ^ 1, b + kTile);
                nValid = rank_tile(sItems, dts, cnt, fuse, q, false, t > 0);
            }
            // consecutive threads write consecutive 16-byte vectors of the
            // destination-grouped tile (coalesced runs per destination)
            const uint32_t total = nValid * V;
            for (uint32_t v = tid; v < total; v += kB) {
                const uint32_t slot = v / V;
                const uint32_t part = v - slot * V;
                const uint32_t dst = slotDst[slot];
                const uint32_t src = slotSrc[slot];
                const uint4 val = sItems[src * V + part];
                if (W::kAppendRetired && (dst & kRetFlag)) {
                    const uint32_t r = dst & ~kRetFlag;
                    if (r < a.retiredCap) a.retiredOut[(size_t)r * V + part] = val;
                } else {
                    nxtItems[(size_t)dst * V + part] = val;
                    if (kFuse && fuse && part == 0u) {
                        const int32_t d2 = dts[src];
                        nxtDest[dst] = d2;
                        const uint32_t dg = digit_of(d2);
                        if (push && dg < (uint32_t)D) {
                            const uint32_t oc = ((uint32_t)G * ((dst & ~15u) + 1u) - 1u) / nNext;
                            atomicAdd(&totNext[(size_t)oc * Dp + dg], 1u);
                            atomicAdd(&grpNext[(size_t)(oc / (uint32_t)grpSize) * Dp + dg], 1u);
                        }
                    }
                }
            }
            // (no barrier: the next tile's wait is the one before this buffer is refilled)
        }
        fence_proxy_async_global();
        if (logRound) {
            a.roundLog[7 * round + 3] = globaltimer();
            a.roundLog[7 * round + 5] = n;
            a.roundLog[7 * round + 6] = nNext;
        }
        if (failed || !round_barrier()) {
            failed = true;
            break;
        }
        if (logRound) a.roundLog[7 * round + 4] = globaltimer();
        if constexpr (HasProgress<W>::value) {
            if (a.progress && c == 0 && tid == 0) {
                // every CTA's sink writes of this round precede the barrier just passed
                __threadfence_system();
                *a.progress = retiredSoFar;
            }
        }
        n = nNext;
        pushed = push;
        fresh = !fuse;
        xsel = fuse ? xsel ^ 1u : 0u;
        if (pre) pre = false;
        else ++round;
    }
    // let any copy still in flight (a prefetch before a failed barrier) land
    if (tid == 0) {
        if (pend0) (void)mbar_wait_bounded(&bar[0], par0);
        if (pend1) (void)mbar_wait_bounded(&bar[1], par1);
    }
    if (a.seedCount && c == 0) {
        // the seeded out-queue has been consumed; with nothing seeded the
        // incoming queue is empty
        if (pre)
            for (int e = tid; e <= R; e += kB) a.inOffset[e] = 0u;
        if (tid == 0) *a.seedCount = 0ull;
    }
    if (c == 0 && tid == 0) {
        a.result[0] = round;
        a.result[1] = forwarded;
        a.result[2] = failed ? RF_DEV_TIMEOUT : 0u;
        a.result[3] = retiredSoFar;
        for (int k = 0; k < K; ++k) a.result[4 + kMaxRuns + k] = sRet[k];
        if (a.retiredCountOut) *a.retiredCountOut = retiredSoFar;
        *a.numActiveOut = failed ? 0ull : n;
    }
}

// Host side: one cooperative launch of rounds_kernel<W> over the context's
// queues, starting from its current incoming queue, or (seeded) from its
// out-queue with the items' first ranks as destinations.  res (host)
// receives {rounds, forwarded, status, retired}.  Waits for the stream.
// numRuns > 1 (seeded, steps on arrival, policies with kAppendRetired): the
// seeded items belong to that many independent runs, named by the high bits
// of their destination words; run k retires into sink slots
// [k runCap, (k + 1) runCap).  runOut (host, nullable, 2 kMaxRuns words)
// receives each run's rounds, then each run's retired count.  progress
// (nullable, device address of host-mapped memory) receives, after every
// round, how many retired items' sink slots are final; poll (nullable) is
// called over and over while the launch runs.
template <class W>
rf_status launch_rounds(rf_ctx *ctx, const W &work, uint32_t maxRounds, cudaStream_t s,
                        unsigned long long *roundLog, uint32_t roundLogCap, uint4 *retiredOut,
                        unsigned long long retiredCap, unsigned long long *retiredCountOut, unsigned long long res[4],
                        bool stepOnArrival = false, bool seeded = false, const void *seedItems = nullptr,
                        uint32_t numRuns = 1, unsigned long long runCap = 0, unsigned long long *runOut = nullptr,
                        unsigned long long *progress = nullptr, const std::function<void()> *poll = nullptr)
{
    if ((seeded || stepOnArrival) && !W::kFuseStep) {
        set_error("persistent rounds: the policy does not step on arrival");
        return RF_ERR_ARG;
    }
    if (seeded && !stepOnArrival) {
        set_error("persistent rounds: a seeded start needs steps on arrival");
        return RF_ERR_ARG;
    }
    if (numRuns < 1 || numRuns > (uint32_t)kMaxRuns ||
        (numRuns > 1 && (!W::kAppendRetired || !seeded || !retiredOut ||
                         (unsigned long long)numRuns * runCap > retiredCap || numRuns * runCap >= (1ull << 31)))) {
        set_error("persistent rounds: %u runs (at most %d, each with its own sink, seeded, steps on arrival)",
                  numRuns, kMaxRuns);
        return RF_ERR_ARG;
    }
    const uint32_t itemBytes = 16u * W::V;
    if (ctx->itemBytes != itemBytes) {
        set_error("persistent rounds: the workload moves %u-byte items, the context %u", itemBytes,
                  ctx->itemBytes);
        return RF_ERR_ARG;
    }
    const int R = ctx->numRanks;
    const int D = R + (W::kAppendRetired ? (int)numRuns : 0);
    if (D > 8 * W::kBlock) {
        set_error("persistent rounds: %d destinations exceed %d", D, 8 * W::kBlock);
        return RF_ERR_ARG;
    }
    const RoundsLayout L = rounds_layout(itemBytes, D, work.smemBytes(), W::kBlock * W::kItemsPerThread, W::kBlock / 32);
    int optin = 0;
    RF_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    auto fn = rounds_kernel<W>;
    cudaFuncAttributes fa;
    RF_CUDA(cudaFuncGetAttributes(&fa, fn));
    const int dynMax = optin - (int)fa.sharedSizeBytes;  // the limit covers static shared memory too
    if ((int)L.total > dynMax) {
        set_error("persistent rounds: %u bytes of shared memory per CTA exceed the device's %d", L.total, dynMax);
        return RF_ERR_ARG;
    }
    RF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dynMax));
    // Shared memory carve-out: just what W::kMinBlocksPerSM CTAs need, so the
    // rest of the SM's on-chip memory stays L1 for the workload's gathers.
    int smPerSM = 0;
    RF_CUDA(cudaDeviceGetAttribute(&smPerSM, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device));
    const long long need = (long long)W::kMinBlocksPerSM * ((long long)L.total + fa.sharedSizeBytes + 1024);
    const int carve = smPerSM > 0 ? (int)((100 * need + smPerSM - 1) / smPerSM) : 100;
    RF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, carve < 100 ? carve : 100));
    int perSM = 0;
    RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perSM, fn, W::kBlock, L.total));
    if (perSM < W::kMinBlocksPerSM) {
        // the hint did not leave room for the intended occupancy: leave the carve-out to CUDA
        RF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, -1));
        RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perSM, fn, W::kBlock, L.total));
    }
    if (perSM < 1) {
        set_error("persistent rounds: the kernel does not fit on an SM");
        return RF_ERR_ARG;
    }
    const int G = ctx->numSMs * perSM;
    const size_t totBytes = (size_t)3 * G * rounds_row_stride(D) * sizeof(uint32_t);
    const size_t grpBytes = (size_t)3 * kSyncGroups * rounds_row_stride(D) * sizeof(uint32_t);
    const size_t smBytes = rounds_align_sz((size_t)G * sizeof(uint32_t), 16);
    const size_t tailBytes = grpBytes + sizeof(GridSync) + kResultWords * sizeof(unsigned long long) + smBytes;
    // second destination array (step on arrival), padded like ctx->dest
    const size_t dest2Bytes = W::kFuseStep ? rounds_align_sz((size_t)(ctx->capacity + 3) / 4 * 16 + 16, 256) : 0;
    if (rf_status st = ensure_rounds_scratch(ctx, rounds_align_sz(totBytes + tailBytes, 256) + dest2Bytes)) return st;
    unsigned char *base = static_cast<unsigned char *>(ctx->roundsScratch);
    RoundsArgs a;
    a.in = static_cast<uint4 *>(ctx->in);
    a.out = static_cast<uint4 *>(ctx->out);
    a.dest = ctx->dest;
    a.inOffset = ctx->inOffset;
    a.tot = reinterpret_cast<uint32_t *>(base);
    a.grpTot = reinterpret_cast<uint32_t *>(base + totBytes);
    a.sync = reinterpret_cast<GridSync *>(base + totBytes + grpBytes);
    a.result = reinterpret_cast<unsigned long long *>(base + totBytes + grpBytes + sizeof(GridSync));
    a.smOf = reinterpret_cast<uint32_t *>(base + totBytes + grpBytes + sizeof(GridSync) +
                                          kResultWords * sizeof(unsigned long long));
    // the SM table is staged in the tile buffers: G + 3 words must fit
    a.skew = W::kFuseStep && ((size_t)G + 3) * 4 <= (size_t)2 * W::kBlock * W::kItemsPerThread * itemBytes
                 ? (ctx->rankSkew < 32u ? ctx->rankSkew : 32u)
                 : 0u;
    a.dest2 = W::kFuseStep ? reinterpret_cast<int32_t *>(base + rounds_align_sz(totBytes + tailBytes, 256)) : nullptr;
    a.numActiveOut = &ctx->dev->numActive;
    a.roundLog = roundLog;
    a.roundLogCap = roundLog ? roundLogCap : 0u;
    a.retiredOut = retiredOut;
    a.retiredCap = retiredOut ? retiredCap : 0ull;
    a.retiredCountOut = retiredCountOut;
    a.seedCount = seeded ? &ctx->dev->outCount : nullptr;
    a.seedItems = seeded ? static_cast<const uint4 *>(seedItems) : nullptr;
    a.fuseStep = stepOnArrival ? 1u : 0u;
    a.spinLimit = ctx->waitLimitCycles ? (long long)ctx->waitLimitCycles : kSpinLimitCycles;
    a.missingArrivals = ctx->missingArrivals;
    // the owner of a pushed count is computed in 32 bits: G x (pushMax + 1) < 2^32
    const uint32_t pushCap = (uint32_t)(0xFFFFFFFFu / (uint32_t)G) - 1u;
    a.pushMax = W::kFuseStep && stepOnArrival ? (ctx->pushMax < pushCap ? ctx->pushMax : pushCap) : 0u;
    a.maxRounds = maxRounds;
    a.numRanks = R;
    a.numRuns = numRuns;
    a.runCap = numRuns > 1 ? (uint32_t)runCap : 0u;
    a.progress = progress;
    RF_CUDA(cudaMemsetAsync(base, 0, totBytes + tailBytes, s));
    W w = work;
    void *params[] = {&a, &w};
    time_begin(ctx, kTimeRounds, s);
    RF_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(fn), dim3(G), dim3(W::kBlock), params,
                                        L.total, s));
    count_launch();
    time_end(ctx, kTimeRounds, s);
    if (poll)  // the caller's work while the launch runs (stream order stays as it is)
        while (cudaStreamQuery(s) == cudaErrorNotReady) (*poll)();
    RF_CUDA(cudaMemcpyAsync(ctx->host, ctx->dev, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    unsigned long long r[kResultWords] = {};
    RF_CUDA(cudaMemcpyAsync(r, a.result, sizeof r, cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaStreamSynchronize(s));
    ctx->pending = false;
    time_collect(ctx);
    for (int i = 0; i < 4; ++i) res[i] = r[i];
    if (runOut)
        for (int i = 0; i < 2 * kMaxRuns; ++i) runOut[i] = r[4 + i];
    if (r[2] & RF_DEV_TIMEOUT) {
        set_error("persistent rounds: a bounded device-side wait gave up");
        return RF_ERR_TIMEOUT;
    }
    return RF_OK;
}

// The shapes a policy compiles, in order: launch number v of them, or list
// them for the host.  Every shape runs the same rounds.
template <class W, class... Ss>
struct ShapeList {
    static constexpr int kCount = sizeof...(Ss);
    static void infos(ShapeInfo *out)
    {
        int i = 0;
        ((out[i++] = ShapeInfo{Ss::kBlock, Ss::kItemsPerThread, Ss::kMinBlocksPerSM}), ...);
    }
    template <class... Args>
    static rf_status launch(int v, rf_ctx *ctx, const W &w, Args &&...args)
    {
        rf_status st = RF_ERR_ARG;
        int i = 0;
        bool done = false;
        // only the chosen shape's launch runs, so each argument is used once
        ((i++ == v ? (st = launch_rounds(ctx, Ss(w), std::forward<Args>(args)...), done = true) : false), ...);
        if (!done) set_error("persistent rounds: shape %d of %d", v, kCount);
        return st;
    }
};

}  // namespace rfi
