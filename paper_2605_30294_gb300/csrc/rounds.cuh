// Batched form of the forwarding loop: every round of "work, then exchange"
// in one persistent cooperative kernel, with no host round trip per round.
//
// The plain loop (Sec. 5.1's "alternate between the render kernel and
// forwardRays until no ray is left") launches a work kernel and the exchange
// kernels per round and reads the active count back on the host.  Here all
// CTAs of one cooperative launch stay resident and run the rounds
// themselves:
//
//   phase 1  each CTA takes a contiguous range of the incoming queue, stages
//            it tile by tile with a bulk async copy, applies the workload's
//            step to every item and writes the tile back to the same slots of
//            the out-queue with one bulk store (destination -1 for an item
//            that retired: the paper's first single-array queue, Sec. 3.2),
//            counting destinations per CTA;
//   barrier  (bounded spin)
//   phase 2  per-destination totals -> segment offsets (Sec. 4.2.2) and the
//            next active count (Sec. 4.2.3); each CTA's base per destination =
//            segment offset + the counts of the CTAs before it;
//   phase 3  each CTA re-reads its range of the out-queue and scatters it,
//            stably and grouped by destination, into the incoming queue;
//   barrier  then the next round, until no item is active.
//
// Because the out slot of an item is its input slot and every step is
// stable, queue order never depends on scheduling: round k's incoming queue
// equals the one of a serial round-by-round simulation.
//
// Every wait is bounded; a wait that gives up raises an abort flag that all
// CTAs check at the next barrier, and the kernel returns with a timeout status.
#pragma once

#include "internal.cuh"
#include "rafi_device.cuh"

namespace rfi {

constexpr int kSyncGroups = 16;  // first level of the grid barrier

struct GridSync {
    unsigned int count;  // groups complete at the current barrier
    unsigned int gen;    // barrier generation
    unsigned int abort;  // set by a CTA whose wait gave up
    unsigned int work[2];  // work-phase chunk counters (round parity), dynamic policies
    unsigned int pad[27];
    unsigned int group[kSyncGroups][32];  // CTAs arrived per group, one 128-byte line each
};

struct RoundsArgs {
    uint4 *in;
    uint4 *out;
    int32_t *dest;             // capacity rounded up to 4 entries + 4 (bulk-copied in 16-byte units)
    uint32_t *inOffset;        // numRanks + 1
    uint32_t *tot;             // gridDim.x rows of per-CTA destination counts (row stride: digits rounded to 4)
    unsigned int *total;       // 2 x digits: per-destination totals (round parity)
    GridSync *sync;
    unsigned long long *result;  // {rounds, forwarded, status, retired}
    unsigned long long *numActiveOut;  // items still active when the kernel returns
    unsigned long long *roundLog;  // nullable: per round {t_start, t_work_end, t_barrier1, t_scatter_end, t_barrier2, n_in, n_next}
    uint4 *retiredOut;         // retirement sink (policies with kAppendRetired)
    unsigned long long retiredCap;
    unsigned long long *retiredCountOut;
    uint32_t maxRounds;
    uint32_t roundLogCap;
    int32_t numRanks;
};

constexpr int kRoundsBlock = 256;
constexpr int kRoundsWarps = kRoundsBlock / 32;
constexpr int kRoundsK = 2;  // items per thread per tile
constexpr uint32_t kRoundsTile = kRoundsBlock * kRoundsK;

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

// Bounded grid barrier for a cooperative launch (all CTAs resident), in two
// levels: CTAs arrive on one of kSyncGroups group counters (separate cache
// lines), the last CTA of a group arrives on the top counter, and the last
// group releases everyone by bumping the generation.
// Returns false when any CTA has given up; the caller must then return.
__device__ inline bool grid_barrier(GridSync *gs, unsigned int *sFlag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int ok = 1;
        const unsigned int g = ld_acquire(&gs->gen);
        const unsigned int G = gridDim.x;
        const unsigned int groups = G < (unsigned)kSyncGroups ? G : (unsigned)kSyncGroups;
        const unsigned int grp = blockIdx.x % groups;
        const unsigned int members = G / groups + (grp < G % groups ? 1u : 0u);
        __threadfence();
        bool last = false;
        if (atomicAdd(&gs->group[grp][0], 1u) + 1u == members) {
            atomicExch(&gs->group[grp][0], 0u);
            __threadfence();
            last = atomicAdd(&gs->count, 1u) + 1u == groups;
        }
        if (last) {
            atomicExch(&gs->count, 0u);
            __threadfence();
            st_release(&gs->gen, g + 1u);
        } else {
            const long long t0 = clock64();
            while (ld_acquire(&gs->gen) == g) {
                if (ld_acquire(&gs->abort)) {
                    ok = 0;
                    break;
                }
                if (clock64() - t0 > kSpinLimitCycles) {
                    atomicExch(&gs->abort, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (ld_acquire(&gs->abort)) ok = 0;
        *sFlag = ok;
    }
    __syncthreads();
    return *sFlag != 0;
}

// Exclusive block scan of v[0..n) in shared memory (n <= 8 * kRoundsBlock).
__device__ inline uint32_t rounds_block_scan(uint32_t *v, int n, uint32_t *tmp)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __syncthreads();
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
        const uint32_t w = lane < kRoundsWarps ? tmp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kRoundsWarps) tmp[lane] = wi - w;
        if (lane == 31) tmp[kRoundsWarps] = wi;
    }
    __syncthreads();
    const uint32_t base = tmp[warp] + incl - sum;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int i = tid * 8 + j;
        if (i < n) v[i] = base + x[j];
    }
    const uint32_t total = tmp[kRoundsWarps];
    __syncthreads();
    return total;
}

struct RoundsLayout {
    uint32_t items, dests, wc, cnt, start, base, tot, off, slotSrc, slotDst, tmp, flag, bar, work, total;
};

__host__ __device__ inline uint32_t rounds_align(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// items: two tile buffers (double buffering); the same bytes stage the
// per-CTA count rows in phase 2.  dests: the tiles' destinations.  D =
// destination digits (ranks, plus one retirement digit when the policy
// appends retired items).
__host__ __device__ inline RoundsLayout rounds_layout(uint32_t itemBytes, int D, uint32_t workBytes,
                                                  uint32_t tile = kRoundsTile)
{
    RoundsLayout L;
    uint32_t o = 0;
    L.items = o;   o = rounds_align(o + 2u * tile * itemBytes, 128);
    L.dests = o;   o = rounds_align(o + 2u * (tile + 4u) * 4u, 16);
    L.wc = o;      o = rounds_align(o + kRoundsWarps * D * 4u, 16);
    L.cnt = o;     o = rounds_align(o + D * 4u, 16);
    L.start = o;   o = rounds_align(o + D * 4u, 16);
    L.base = o;    o = rounds_align(o + D * 4u, 16);
    L.tot = o;     o = rounds_align(o + D * 4u, 16);
    L.off = o;     o = rounds_align(o + (D + 1) * 4u, 16);
    L.slotSrc = o; o = rounds_align(o + tile * 2u, 16);
    L.slotDst = o; o = rounds_align(o + tile * 4u, 16);
    L.tmp = o;     o = rounds_align(o + (kRoundsWarps + 1) * 4u, 16);
    L.flag = o;    o = rounds_align(o + 4u, 16);
    L.bar = o;     o = rounds_align(o + 16u, 16);
    L.work = o;    o = rounds_align(o + workBytes, 16);
    L.total = o;
    return L;
}

// The workload policy W provides:
//   static constexpr int V;               16-byte vectors per item
//   static constexpr bool kAppendRetired; retired items go, stably, to the
//                                         retirement sink (else: retire())
//   static constexpr bool kDynamicWork;   long, uneven per-item work: the work
//                                         phase hands out chunks dynamically
//   static constexpr int kMinBlocksPerSM; resident CTAs per SM to compile for
//   static constexpr int kItemsPerThread; tile = 256 x this many items
//   uint32_t smemBytes() const;           its own shared memory
//   void load_smem(void *s) const;        fill it (all threads; a barrier follows)
//   int32_t step(uint4 (&w)[V], int32_t rank, uint32_t round, const void *s) const;
//       advances one item: returns the destination rank (w updated) or -1 to retire
//   void retire(const uint4 (&w)[V]) const;  (used when !kAppendRetired)
template <class W>
__global__ void __launch_bounds__(kRoundsBlock, W::kMinBlocksPerSM) rounds_kernel(RoundsArgs a, W work)
{
    constexpr int V = W::V;
    constexpr uint32_t kItemBytes = 16u * V;
    constexpr int kK = W::kItemsPerThread;  // items per thread per tile
    constexpr uint32_t kTile = kRoundsBlock * kK;
    constexpr uint32_t kTileVecs = kTile * V;
    constexpr uint32_t kRetFlag = 0x80000000u;
    extern __shared__ __align__(128) unsigned char smem[];
    const int R = a.numRanks;
    const int D = R + (W::kAppendRetired ? 1 : 0);  // digits: ranks (+ retirement)
    const int Dp = rounds_row_stride(D);
    const RoundsLayout L = rounds_layout(kItemBytes, D, work.smemBytes(), kTile);
    uint4 *sBuf = reinterpret_cast<uint4 *>(smem + L.items);  // two tiles of kTileVecs
    uint32_t *sRows = reinterpret_cast<uint32_t *>(smem + L.items);
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
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);  // bar[0], bar[1]: one per tile buffer
    void *sWork = smem + L.work;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, c = blockIdx.x;
    const int nbits = 32 - __clz(D);  // keys 0..D (D = no item)
    const uint32_t rowsPerStage = (2u * kTileVecs * 16u) / (uint32_t)(Dp * 4);

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async_smem();
    }
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
    // Once a round is this small, CTA 0 finishes the run alone: the other CTAs
    // return and the round barriers become block barriers.
    constexpr uint32_t kSoloItems = 2u * kTile;
    bool solo = false;
    auto round_barrier = [&]() -> bool {
        if (!solo) return grid_barrier(a.sync, sFlag);
        __threadfence();
        __syncthreads();
        return true;
    };

    uint32_t n = a.inOffset[R];
    unsigned long long forwarded = 0, retiredSoFar = 0;
    uint32_t round = 0;
    bool failed = false;

    for (;; ++round) {
        if (n == 0 || round >= a.maxRounds) break;
        if (!solo && n <= kSoloItems) {
            solo = true;
            if (c != 0) break;
        }
        const int g = solo ? 1 : G;
        const bool logRound = a.roundLog && c == 0 && tid == 0 && round < a.roundLogCap;
        if (logRound) a.roundLog[7 * round + 0] = globaltimer();
        for (int e = tid; e <= R; e += kRoundsBlock) sOff[e] = a.inOffset[e];
        for (int e = tid; e < D; e += kRoundsBlock) sTot[e] = 0u;
        __syncthreads();
        const uint32_t lo = bound(n, c, g);
        const uint32_t hi = bound(n, c + 1, g);
        const uint32_t nt = (hi - lo + kTile - 1) / kTile;

        // ---- phase 1: work step, write back to the same slots ------------------
        // Policies with long, uneven per-item work (W::kDynamicWork) take
        // 32-item chunks from a round counter instead of a fixed range; each
        // CTA then counts its own range's destinations after the barrier.
        const bool dynamic = W::kDynamicWork && !solo;
        if (dynamic) {
            unsigned int *ticket = &a.sync->work[round & 1u];
            for (;;) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(ticket, 32u);
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
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
            if (c == 0 && tid == 0) a.sync->work[(round + 1u) & 1u] = 0u;  // next round's counter
        }
        if (!dynamic && tid == 0 && nt) {
            const uint32_t cnt0 = min(kTile, hi - lo);
            issue_bytes(0, sBuf, a.in + (size_t)lo * V, cnt0 * kItemBytes, nullptr, nullptr, 0u);
        }
        for (uint32_t t = 0; !dynamic && t < nt; ++t) {
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
                const uint32_t j = (uint32_t)(k * kRoundsBlock + tid);
                const bool valid = j < cnt;
                int32_t d = -1;
                if (valid) {
                    uint4 w[V];
#pragma unroll
                    for (int q = 0; q < V; ++q) w[q] = sItems[j * V + q];
                    const int32_t rank = rf::rankOf(sOff, R, b + j);
                    d = work.step(w, rank, round, sWork);
                    if (d >= 0) {
#pragma unroll
                        for (int q = 0; q < V; ++q) sItems[j * V + q] = w[q];
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
        if (logRound) a.roundLog[7 * round + 1] = globaltimer();
        if (dynamic) {
            fence_proxy_async_global();
            if (!round_barrier()) {
                failed = true;
                break;
            }
            // count the destinations of this CTA's range
            for (uint32_t b = lo; b < hi; b += kRoundsBlock) {
                const uint32_t i = b + tid;
                const int32_t d = i < hi ? __ldcg(a.dest + i) : -1;
                const int key = (uint32_t)d < (uint32_t)D ? d : D;
                const unsigned peers = peers_of(key, nbits);
                if (key < D && lane == __ffs(peers) - 1) atomicAdd(&sTot[key], (uint32_t)__popc(peers));
            }
            __syncthreads();
        }
        if (!failed) {
            for (int e = tid; e < D; e += kRoundsBlock) {
                const uint32_t v = sTot[e];
                a.tot[(size_t)c * Dp + e] = v;
                if (v) atomicAdd(&a.total[(round & 1u) * D + e], v);
            }
        }
        fence_proxy_async_global();
        if (failed || !round_barrier()) {
            failed = true;
            break;
        }
        if (logRound) a.roundLog[7 * round + 2] = globaltimer();

        // ---- phase 2: offsets, next count, this CTA's base per destination -----
        for (int e = tid; e < D; e += kRoundsBlock) {
            dStart[e] = a.total[(round & 1u) * D + e];
            dBase[e] = 0u;
        }
        const uint32_t retiredNow = W::kAppendRetired ? a.total[(round & 1u) * D + R] : 0u;
        const uint32_t nNext = rounds_block_scan(dStart, R, tmp);  // ranks only
        if (W::kAppendRetired && tid == 0) dStart[R] = (uint32_t)retiredSoFar;
        {
            // counts of CTAs 0 .. c-1, staged a block of rows at a time
            const int groups = D >= kRoundsBlock ? 1 : kRoundsBlock / D;
            // (a CTA with nothing to scatter needs no base)
            const uint32_t rowsNeeded = nt ? (uint32_t)c : 0u;
            for (uint32_t r0 = 0; r0 < rowsNeeded && !failed; r0 += rowsPerStage) {
                const uint32_t rows = min(rowsPerStage, rowsNeeded - r0);
                if (tid == 0) issue_bytes(0, sRows, a.tot + (size_t)r0 * Dp, rows * Dp * 4u, nullptr, nullptr, 0u);
                if (!wait(0)) {
                    failed = true;
                    break;
                }
                for (int t = tid; t < groups * D; t += kRoundsBlock) {
                    const int e = t % D, g = t / D;
                    uint32_t sum = 0;
                    for (uint32_t rr = g; rr < rows; rr += groups) sum += sRows[rr * Dp + e];
                    if (sum) atomicAdd(&dBase[e], sum);
                }
                __syncthreads();
            }
            __syncthreads();
            for (int e = tid; e < D; e += kRoundsBlock) dBase[e] += dStart[e];
        }
        if (c == 0) {
            for (int e = tid; e < R; e += kRoundsBlock) a.inOffset[e] = dStart[e];
            for (int e = tid; e < D; e += kRoundsBlock) a.total[((round + 1u) & 1u) * D + e] = 0u;
            if (tid == 0) a.inOffset[R] = nNext;
        }
        forwarded += nNext;
        retiredSoFar += retiredNow;
        __syncthreads();

        // ---- phase 3: stable scatter of this CTA's range -----------------------
        auto issue3 = [&](int buf, uint32_t bb) {
            const uint32_t cc = min(kTile, hi - bb);
            issue_bytes(buf, sBuf + buf * kTileVecs, a.out + (size_t)bb * V, cc * kItemBytes,
                        sDst + buf * (kTile + 4u), a.dest + bb, ((cc + 3u) & ~3u) * 4u);
        };
        if (tid == 0 && nt && !failed) issue3(0, lo);
        for (uint32_t t = 0; t < nt && !failed; ++t) {
            const int buf = t & 1;
            const uint32_t b = lo + t * kTile;
            const uint32_t cnt = min(kTile, hi - b);
            if (tid == 0 && t + 1 < nt) issue3(buf ^ 1, b + kTile);
            for (int e = lane; e < D; e += 32) wc[warp * D + e] = 0u;
            if (!wait(buf)) {
                failed = true;
                break;
            }
            const int32_t *dts = sDst + buf * (kTile + 4u);
            int myD[kK];
            uint32_t myR[kK];
#pragma unroll
            for (int k = 0; k < kK; ++k) {
                const uint32_t idx = (uint32_t)(warp * 32 * kK + k * 32 + lane);
                const int32_t d = idx < cnt ? dts[idx] : -1;
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
            }
            __syncthreads();
            for (int e = tid; e < D; e += kRoundsBlock) {
                uint32_t sum = 0;
#pragma unroll
                for (int ww = 0; ww < kRoundsWarps; ++ww) {
                    const uint32_t v = wc[ww * D + e];
                    wc[ww * D + e] = sum;
                    sum += v;
                }
                dCnt[e] = sum;
                dStart[e] = sum;
            }
            const uint32_t nValid = rounds_block_scan(dStart, D, tmp);
#pragma unroll
            for (int k = 0; k < kK; ++k) {
                if (myD[k] >= 0) {
                    const int d = myD[k];
                    const uint32_t within = wc[warp * D + d] + myR[k];
                    const uint32_t slot = dStart[d] + within;
                    slotSrc[slot] = (uint16_t)(warp * 32 * kK + k * 32 + lane);
                    slotDst[slot] = (dBase[d] + within) | (W::kAppendRetired && d == R ? kRetFlag : 0u);
                }
            }
            __syncthreads();
            const uint4 *sItems = sBuf + buf * kTileVecs;
            const uint32_t total = nValid * V;
            for (uint32_t v = tid; v < total; v += kRoundsBlock) {
                const uint32_t slot = v / V;
                const uint32_t part = v - slot * V;
                const uint32_t dst = slotDst[slot];
                const uint4 val = sItems[(uint32_t)slotSrc[slot] * V + part];
                if (W::kAppendRetired && (dst & kRetFlag)) {
                    const uint32_t r = dst & ~kRetFlag;
                    if (r < a.retiredCap) a.retiredOut[(size_t)r * V + part] = val;
                } else {
                    a.in[(size_t)dst * V + part] = val;
                }
            }
            __syncthreads();
            for (int e = tid; e < D; e += kRoundsBlock) dBase[e] += dCnt[e];
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
        n = nNext;
    }
    if (c == 0 && tid == 0) {
        a.result[0] = round;
        a.result[1] = forwarded;
        a.result[2] = failed ? RF_DEV_TIMEOUT : 0u;
        a.result[3] = retiredSoFar;
        if (a.retiredCountOut) *a.retiredCountOut = retiredSoFar;
        *a.numActiveOut = failed ? 0ull : n;
    }
}

// Host side: one cooperative launch of rounds_kernel<W> over the context's
// queues, starting from its current incoming queue.  res (host) receives
// {rounds, forwarded, status, 0}.  Waits for the stream.
template <class W>
rf_status launch_rounds(rf_ctx *ctx, const W &work, uint32_t maxRounds, cudaStream_t s,
                        unsigned long long *roundLog, uint32_t roundLogCap, uint4 *retiredOut,
                        unsigned long long retiredCap, unsigned long long *retiredCountOut, unsigned long long res[4])
{
    const uint32_t itemBytes = 16u * W::V;
    if (ctx->itemBytes != itemBytes) {
        set_error("persistent rounds: the workload moves %u-byte items, the context %u", itemBytes,
                  ctx->itemBytes);
        return RF_ERR_ARG;
    }
    const int R = ctx->numRanks;
    const int D = R + (W::kAppendRetired ? 1 : 0);
    if (D > 8 * kRoundsBlock) {
        set_error("persistent rounds: %d destinations exceed %d", D, 8 * kRoundsBlock);
        return RF_ERR_ARG;
    }
    const RoundsLayout L = rounds_layout(itemBytes, D, work.smemBytes(), kRoundsBlock * W::kItemsPerThread);
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
    int perSM = 0;
    RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perSM, fn, kRoundsBlock, L.total));
    if (perSM < 1) {
        set_error("persistent rounds: the kernel does not fit on an SM");
        return RF_ERR_ARG;
    }
    const int G = ctx->numSMs * perSM;
    const size_t totBytes = (size_t)G * rounds_row_stride(D) * sizeof(uint32_t);
    const size_t totalBytes = (size_t)2 * D * sizeof(unsigned int);
    const size_t tailBytes = totalBytes + sizeof(GridSync) + 4 * sizeof(unsigned long long);
    if (rf_status st = ensure_rounds_scratch(ctx, totBytes + tailBytes)) return st;
    unsigned char *base = static_cast<unsigned char *>(ctx->roundsScratch);
    RoundsArgs a;
    a.in = static_cast<uint4 *>(ctx->in);
    a.out = static_cast<uint4 *>(ctx->out);
    a.dest = ctx->dest;
    a.inOffset = ctx->inOffset;
    a.tot = reinterpret_cast<uint32_t *>(base);
    a.total = reinterpret_cast<unsigned int *>(base + totBytes);
    a.sync = reinterpret_cast<GridSync *>(base + totBytes + totalBytes);
    a.result = reinterpret_cast<unsigned long long *>(base + totBytes + totalBytes + sizeof(GridSync));
    a.numActiveOut = &ctx->dev->numActive;
    a.roundLog = roundLog;
    a.roundLogCap = roundLog ? roundLogCap : 0u;
    a.retiredOut = retiredOut;
    a.retiredCap = retiredOut ? retiredCap : 0ull;
    a.retiredCountOut = retiredCountOut;
    a.maxRounds = maxRounds;
    a.numRanks = R;
    RF_CUDA(cudaMemsetAsync(base + totBytes, 0, tailBytes, s));
    W w = work;
    void *params[] = {&a, &w};
    time_begin(ctx, kTimeRounds, s);
    RF_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(fn), dim3(G), dim3(kRoundsBlock), params,
                                        L.total, s));
    count_launch();
    time_end(ctx, kTimeRounds, s);
    RF_CUDA(cudaMemcpyAsync(ctx->host, ctx->dev, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    unsigned long long r[4] = {0, 0, 0, 0};
    RF_CUDA(cudaMemcpyAsync(r, a.result, sizeof r, cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaStreamSynchronize(s));
    ctx->pending = false;
    time_collect(ctx);
    for (int i = 0; i < 4; ++i) res[i] = r[i];
    if (r[2] & RF_DEV_TIMEOUT) {
        set_error("persistent rounds: a bounded device-side wait gave up");
        return RF_ERR_TIMEOUT;
    }
    return RF_OK;
}

}  // namespace rfi
