// Forwarding microbenchmark: 64-byte work items that hop between logical
// ranks until they retire.  This is the synthetic stand-in for the paper's
// forwarding-only bandwidth benchmark (Sec. 6.1), driven through the same
// interface an application uses (Sec. 3.3, 3.4): a seed kernel emits the
// initial items (the raygen step of Sec. 5.1), a per-rank work kernel reads
// its incoming segment and forwards or retires each item, and rf_exchange
// delivers the forwarded items, round after round, until none is active.
//
// Hop rule (item words w0..w15): r = Philox4x32-10(key {seed, 1}, counter
// {w0, w1, w15, hop}); r0 < ceil(0.1 * 2^32) retires the item, otherwise r1
// picks the destination d (uniform, Zipf table, or one of the 6 torus
// neighbours of the item's rank) and the item becomes w14 = d, w13 ^= r2,
// w15 += 1.  Philox4x32-10 follows Salmon et al., SC'11.
//
// Forms: the host loop (rf_c1_run), its kernels in a CUDA graph
// (rf_c1_run_graph), one persistent launch per run (rf_c1_run_batched) and
// several independent runs, each with its own law, in one persistent launch
// (rf_c1_run_batched_runs; from page-locked host buffers, one launch per run
// with the host link's two directions pipelined).
#include <cmath>
#include <vector>

#include <chrono>
#include <functional>
#include <thread>

#include "internal.cuh"
#include "philox.cuh"
#include "rafi_device.cuh"
#include "rounds.cuh"

namespace rfi {

namespace {

constexpr int kBlock = 256;
constexpr uint32_t kRetire = 429496730u;  // ceil(0.1 * 2^32)

struct WorkArgs {
    rf_device_queues q;
    const uint32_t *zipfThr;
    uint4 *retired;
    unsigned long long *retiredCount;
    unsigned long long retiredCap;
    uint32_t seed, hop;
    int32_t mode, gx, gy, gz;
    const unsigned long long *hopPtr;  // nullable: the hop (round) comes from the device (graph loop)
};

// Neighbour k of rank src on the gx x gy x gz torus (rank = x + gx (y + gy z)):
// k = 0..5 for +x, -x, +y, -y, +z, -z, wrapping.
__device__ __forceinline__ int32_t torus_neighbour(int32_t src, int32_t k, int32_t gx, int32_t gy, int32_t gz)
{
    int32_t x = src % gx, y = (src / gx) % gy, z = src / (gx * gy);
    if (k == 0) x = (x + 1) % gx;
    else if (k == 1) x = (x + gx - 1) % gx;
    else if (k == 2) y = (y + 1) % gy;
    else if (k == 3) y = (y + gy - 1) % gy;
    else if (k == 4) z = (z + 1) % gz;
    else z = (z + gz - 1) % gz;
    return x + gx * (y + gy * z);
}

__device__ __forceinline__ int32_t choose_dest(int32_t mode, int32_t src, uint32_t r1, int32_t R,
                                               const uint32_t *thr, int32_t gx, int32_t gy, int32_t gz)
{
    if (mode == RF_C1_UNIFORM) return (int32_t)(((unsigned long long)r1 * (unsigned)R) >> 32);
    if (mode == RF_C1_ZIPF) {
        // first k with r1 < thr[k] (thresholds ascending); R - 1 if none
        int32_t lo = 0, hi = R - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (r1 < thr[mid]) hi = mid;
            else lo = mid + 1;
        }
        return lo;
    }
    return torus_neighbour(src, (int32_t)(((unsigned long long)r1 * 6u) >> 32), gx, gy, gz);
}

// Per-rank work kernel.  Each thread takes kWorkItems incoming items per pass
// (base + u * kBlock + tid: a warp reads 32 consecutive items for each u), so
// four items' loads are in flight per thread; the owning rank comes from the
// segment offsets.  DET: out slot = incoming index (retired slots get
// destination -1).  Otherwise forwarded items are appended to the out-queue.
// Retired items are appended to the retirement buffer in both modes.  A pass
// reserves its forwarded and retired slots together: one block scan of the
// warps' two counts, then both atomic adds at once, so the pass waits for one
// atomic round trip.
constexpr int kWorkItems = 4;

template <bool DET>
__global__ void __launch_bounds__(kBlock) work_kernel(WorkArgs a)
{
    constexpr int kWarps = kBlock / 32;
    __shared__ uint32_t sOff[RF_MAX_RANKS + 1];
    __shared__ uint32_t sThr[RF_MAX_RANKS];
    __shared__ uint32_t sWarpF[kWarps], sWarpR[kWarps];
    __shared__ unsigned long long sBaseF, sBaseR;
    const int R = a.q.numRanks;
    for (int e = threadIdx.x; e <= R; e += kBlock) sOff[e] = a.q.inOffset[e];
    if (a.mode == RF_C1_ZIPF)
        for (int e = threadIdx.x; e < R - 1; e += kBlock) sThr[e] = a.zipfThr[e];
    __syncthreads();
    const uint32_t n = sOff[R];
    const uint32_t hop = a.hopPtr ? (uint32_t)*a.hopPtr : a.hop;
    if (DET && blockIdx.x == 0 && threadIdx.x == 0) *a.q.outCount = n;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;

    const uint4 *inq = static_cast<const uint4 *>(a.q.in);
    uint4 *outq = static_cast<uint4 *>(a.q.out);
    constexpr uint32_t kPass = kBlock * kWorkItems;
    for (uint32_t base = blockIdx.x * kPass; base < n; base += gridDim.x * kPass) {
        uint4 w[kWorkItems][4];
        int32_t d[kWorkItems];
        bool act[kWorkItems], ret[kWorkItems];
#pragma unroll
        for (int u = 0; u < kWorkItems; ++u) {
            const uint32_t i = base + (uint32_t)u * kBlock + threadIdx.x;
            act[u] = i < n;
#pragma unroll
            for (int q = 0; q < 4; ++q) w[u][q] = act[u] ? __ldg(inq + (size_t)i * 4 + q) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < kWorkItems; ++u) {
            const uint32_t i = base + (uint32_t)u * kBlock + threadIdx.x;
            ret[u] = false;
            d[u] = -1;
            if (act[u]) {
                const uint4 r = philox4x32_10(make_uint4(w[u][0].x, w[u][0].y, w[u][3].w, hop), make_uint2(a.seed, 1u));
                if (r.x < kRetire) {
                    ret[u] = true;
                } else {
                    d[u] = choose_dest(a.mode, rf::rankOf(sOff, R, i), r.y, R, sThr, a.gx, a.gy, a.gz);
                    w[u][3].z = (uint32_t)d[u];
                    w[u][3].y ^= r.z;
                    w[u][3].w += 1u;
                }
            }
        }
        // per-item ranks within the warp (item index u first, then lane) and the
        // warp's counts, for the appended forwards (not in DET) and retirements
        const uint32_t lt = lanemask_lt();
        uint32_t rankF[kWorkItems], rankR[kWorkItems], cf = 0, cr = 0;
#pragma unroll
        for (int u = 0; u < kWorkItems; ++u) {
            const uint32_t bf = __ballot_sync(0xFFFFFFFFu, !DET && act[u] && !ret[u]);
            const uint32_t br = __ballot_sync(0xFFFFFFFFu, act[u] && ret[u]);
            rankF[u] = cf + (uint32_t)__popc(bf & lt);
            rankR[u] = cr + (uint32_t)__popc(br & lt);
            cf += (uint32_t)__popc(bf);
            cr += (uint32_t)__popc(br);
        }
        if (lane == 0) {
            sWarpF[warp] = cf;
            sWarpR[warp] = cr;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const uint32_t vf = lane < (unsigned)kWarps ? sWarpF[lane] : 0u;
            const uint32_t vr = lane < (unsigned)kWarps ? sWarpR[lane] : 0u;
            uint32_t inF = vf, inR = vr;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t tf = __shfl_up_sync(0xFFFFFFFFu, inF, o);
                const uint32_t tr = __shfl_up_sync(0xFFFFFFFFu, inR, o);
                if ((int)lane >= o) {
                    inF += tf;
                    inR += tr;
                }
            }
            if (lane < (unsigned)kWarps) {
                sWarpF[lane] = inF - vf;
                sWarpR[lane] = inR - vr;
            }
            if (lane == 31) {
                // both reservations in flight at once
                const unsigned long long bF = inF ? atomicAdd(a.q.outCount, (unsigned long long)inF) : 0ull;
                const unsigned long long bR = inR ? atomicAdd(a.retiredCount, (unsigned long long)inR) : 0ull;
                sBaseF = bF;
                sBaseR = bR;
            }
        }
        __syncthreads();
        const unsigned long long baseF = sBaseF + sWarpF[warp], baseR = sBaseR + sWarpR[warp];
#pragma unroll
        for (int u = 0; u < kWorkItems; ++u) {
            if (!act[u]) continue;
            const uint32_t i = base + (uint32_t)u * kBlock + threadIdx.x;
            if (ret[u]) {
                const unsigned long long rs = baseR + rankR[u];
                if (rs < a.retiredCap) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) a.retired[(size_t)rs * 4 + q] = w[u][q];
                }
                if (DET) a.q.dest[i] = -1;
            } else {
                const unsigned long long slot = DET ? (unsigned long long)i : baseF + rankF[u];
                if (slot < a.q.capacity) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) outq[(size_t)slot * 4 + q] = w[u][q];
                    a.q.dest[slot] = d[u];
                }
            }
        }
        __syncthreads();  // the shared counts are rewritten by the next pass
    }
}

// The hop rule as a workload policy of the persistent round kernel
// (rounds.cuh): same arithmetic as work_kernel, one item at a time.  Retired
// items go to the kernel's retirement sink.
struct C1Work {
    static constexpr int V = 4;
    static constexpr bool kAppendRetired = true;
    static constexpr bool kDynamicWork = false;
    static constexpr bool kGridStride = false;
    static constexpr bool kFuseStep = true;
    static constexpr int kMinBlocksPerSM = 3;
    static constexpr int kItemsPerThread = 2;
    static constexpr int kBlock = kRoundsBlock;
    static constexpr unsigned kStepReadMask = 0x9u;   // the step reads words 0-1 and 12-15
    static constexpr unsigned kStepWriteMask = 0x8u;  // and writes words 13-15
    const uint32_t *zipfThr;
    uint32_t seed;
    int32_t mode, gx, gy, gz, R;
    // A launch of several independent runs (runs > 1): run k's law in bits
    // 2k, 2k + 1 of laws, the run in the high bits of each destination word.
    int32_t runs = 1;
    uint32_t laws = 0;
    int32_t lgx = -1, lgy = -1;  // log2 of gx, gy when gx, gy and gz are powers of two (else -1)

    __host__ __device__ int32_t lawOf(uint32_t run) const
    {
        return runs > 1 ? (int32_t)((laws >> (2u * run)) & 3u) : mode;
    }
    __host__ __device__ bool anyLaw(int32_t m) const
    {
        for (int32_t k = 0; k < runs; ++k)
            if (lawOf((uint32_t)k) == m) return true;
        return false;
    }
    // shared memory: the Zipf thresholds (up to 256 ranks followed by a guide of
    // 256 byte entries: guide[b] = the destination of r1 = b 2^24, the first
    // threshold above it), or (up to 256 ranks, one run) the torus neighbour
    // table [rank][6] in bytes; small enough to keep three CTAs per SM (a launch
    // of several runs computes torus neighbours instead of keeping the table)
    __host__ __device__ bool nbrTable() const { return runs <= 1 && mode == RF_C1_NBR6 && R <= 256; }
    __host__ __device__ bool zipfGuide() const { return anyLaw(RF_C1_ZIPF) && R <= 256; }
    __host__ __device__ uint32_t thrBytes() const { return ((uint32_t)(R > 1 ? R - 1 : 1) * 4u + 15u) / 16u * 16u; }
    __host__ __device__ uint32_t smemBytes() const
    {
        return nbrTable() ? ((uint32_t)R * 6u + 15u) / 16u * 16u
                          : (zipfGuide() ? thrBytes() + 256u : (uint32_t)(R > 1 ? R : 1) * 4u);
    }
    __device__ void load_smem(void *s) const
    {
        if (anyLaw(RF_C1_ZIPF)) {
            uint32_t *t = static_cast<uint32_t *>(s);
            for (int e = threadIdx.x; e < R - 1; e += blockDim.x) t[e] = zipfThr[e];
            if (zipfGuide()) {
                uint8_t *g = static_cast<uint8_t *>(s) + thrBytes();
                for (int b = threadIdx.x; b < 256; b += blockDim.x)
                    g[b] = (uint8_t)choose_dest(RF_C1_ZIPF, 0, (uint32_t)b << 24, R, zipfThr, gx, gy, gz);
            }
        }
        if (nbrTable()) {
            uint8_t *t = static_cast<uint8_t *>(s);
            for (int e = threadIdx.x; e < 6 * R; e += blockDim.x)
                t[e] = (uint8_t)torus_neighbour(e / 6, e % 6, gx, gy, gz);
        }
    }
    // word: the item's destination word (its current rank; with several runs,
    // the run in the high bits); returns the next one (same run) or -1
    __device__ int32_t step(uint4 (&w)[4], int32_t word, uint32_t round, const void *s) const
    {
        const uint4 r = philox4x32_10(make_uint4(w[0].x, w[0].y, w[3].w, round), make_uint2(seed, 1u));
        if (r.x < kRetire) return -1;
        const uint32_t run = (uint32_t)word >> 16;
        const int32_t rank = word & 0xFFFF;
        const int32_t law = lawOf(run);
        int32_t d;
        if (law == RF_C1_NBR6 && nbrTable()) {
            d = (int32_t)static_cast<const uint8_t *>(s)[rank * 6 + (int32_t)(((unsigned long long)r.y * 6u) >> 32)];
        } else if (law == RF_C1_NBR6 && lgx >= 0) {
            // power-of-two torus: coordinates by shifts and masks
            const int32_t k = (int32_t)(((unsigned long long)r.y * 6u) >> 32);
            int32_t x = rank & (gx - 1), y = (rank >> lgx) & (gy - 1), z = rank >> (lgx + lgy);
            const int32_t dir = (k & 1) ? -1 : 1;
            if (k < 2) x = (x + dir) & (gx - 1);
            else if (k < 4) y = (y + dir) & (gy - 1);
            else z = (z + dir) & (gz - 1);
            d = x | (y << lgx) | (z << (lgx + lgy));
        } else if (law == RF_C1_ZIPF && R <= 256) {  // the guide is loaded whenever a run is Zipf
            // start at the destination of the bucket's lowest r1 and walk up the
            // (ascending) thresholds: the first k with r1 < thr[k], or R - 1
            const uint32_t *t = static_cast<const uint32_t *>(s);
            d = static_cast<const uint8_t *>(s)[thrBytes() + (r.y >> 24)];
            while (d < R - 1 && r.y >= t[d]) ++d;
        } else {
            d = choose_dest(law, rank, r.y, R, static_cast<const uint32_t *>(s), gx, gy, gz);
        }
        w[3].z = (uint32_t)d;
        w[3].y ^= r.z;
        w[3].w += 1u;
        return d | (int32_t)(run << 16);
    }
    __device__ void retire(const uint4 (&)[4]) const {}
};

// Shapes of the persistent kernel for the microbenchmark (the autotuner's
// candidates): {items per thread, CTAs per SM, threads}; tiles of 512, 768
// and 1024 items (the larger the tile, the longer each destination's run of
// stores), one shape per SM-occupancy that fits the tile's shared memory.
using C1Shapes = ShapeList<C1Work, Shape<C1Work, 2, 3, 256>, Shape<C1Work, 3, 2, 256>, Shape<C1Work, 4, 1, 256>,
                           Shape<C1Work, 2, 1, 512>>;

// The same policy publishing its retired count after every round, for the
// runs whose retired items leave for the host while the launch still runs.
struct C1WorkProgress : C1Work {
    static constexpr bool kProgress = true;
    C1WorkProgress() = default;
    __host__ __device__ explicit C1WorkProgress(const C1Work &w) : C1Work(w) {}
};
using C1ProgressShapes =
    ShapeList<C1WorkProgress, Shape<C1WorkProgress, 2, 3, 256>, Shape<C1WorkProgress, 3, 2, 256>,
              Shape<C1WorkProgress, 4, 1, 256>, Shape<C1WorkProgress, 2, 1, 512>>;

// Seed: emit item i to rank i mod R at out slot base + i, where base was
// reserved on the append counter by reserve_kernel.
__global__ void __launch_bounds__(kBlock) seed_kernel(const uint4 *items, uint32_t n, rf_device_queues q,
                                                      const unsigned long long *base)
{
    const unsigned long long b = *base;
    uint4 *outq = static_cast<uint4 *>(q.out);
    const uint64_t vecs = (uint64_t)n * 4u;
    for (uint64_t v = blockIdx.x * (uint64_t)kBlock + threadIdx.x; v < vecs; v += (uint64_t)gridDim.x * kBlock) {
        const uint32_t i = (uint32_t)(v >> 2);
        if (b + i < q.capacity) {
            outq[(b + i) * 4 + (v & 3u)] = __ldg(items + v);
            if ((v & 3u) == 0) q.dest[b + i] = (int32_t)(i % (uint32_t)q.numRanks);
        }
    }
}

// Seed for items already copied into out slots [0, n): destinations only.
__global__ void __launch_bounds__(kBlock) seed_dest_kernel(uint32_t n, rf_device_queues q)
{
    for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock)
        q.dest[i] = (int32_t)(i % (uint32_t)q.numRanks);
    if (blockIdx.x == 0 && threadIdx.x == 0) *q.outCount = n;
}

// Seed for several runs' items copied (or read in place) as one array of
// numRuns x n: item i of run k, at slot k n + i, starts at rank i mod R, with
// the run in the high bits of its destination word.
__global__ void __launch_bounds__(kBlock) seed_dest_runs_kernel(uint32_t total, uint32_t n, rf_device_queues q)
{
    for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < total; i += gridDim.x * kBlock)
        q.dest[i] = (int32_t)(((i / n) << 16) | ((i % n) % (uint32_t)q.numRanks));
    if (blockIdx.x == 0 && threadIdx.x == 0) *q.outCount = total;
}

__global__ void reserve_kernel(unsigned long long *counter, unsigned long long n, unsigned long long *base)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *base = atomicAdd(counter, n);
}

rf_status check_c1(rf_ctx *ctx, const char *fn)
{
    if (!ctx) {
        set_error("%s: NULL context", fn);
        return RF_ERR_ARG;
    }
    if (ctx->itemBytes != 64) {
        set_error("%s: the microbenchmark moves 64-byte items (context has %u)", fn, ctx->itemBytes);
        return RF_ERR_ARG;
    }
    return RF_OK;
}

rf_status ensure_zipf(rf_ctx *ctx, double s)
{
    if (ctx->zipfS == s) return RF_OK;
    std::vector<uint32_t> thr((size_t)ctx->numRanks, 0u);
    rf_status st = rf_c1_zipf_thresholds(ctx->numRanks, s, thr.data());
    if (st != RF_OK) return st;
    RF_CUDA(cudaMemcpy(ctx->zipfThr, thr.data(), thr.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    ctx->zipfS = s;
    return RF_OK;
}

int grid_for(rf_ctx *ctx, uint64_t work, int perSM)
{
    const uint64_t want = (work + kBlock - 1) / kBlock;
    const uint64_t cap = (uint64_t)ctx->numSMs * (uint64_t)perSM;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace
}  // namespace rfi

using namespace rfi;

extern "C" {

rf_status rf_c1_zipf_thresholds(int32_t numRanks, double s, uint32_t *thrHost)
{
    if (numRanks < 1 || numRanks > RF_MAX_RANKS || !thrHost || !(s > 0.0)) {
        set_error("rf_c1_zipf_thresholds: bad arguments");
        return RF_ERR_ARG;
    }
    double total = 0.0;
    for (int32_t j = 1; j <= numRanks; ++j) total += std::pow((double)j, -s);
    double partial = 0.0;
    for (int32_t k = 0; k + 1 < numRanks; ++k) {
        partial += std::pow((double)(k + 1), -s);
        thrHost[k] = (uint32_t)std::floor(partial / total * 4294967296.0);
    }
    return RF_OK;
}

rf_status rf_c1_seed(rf_ctx *ctx, const void *items, uint64_t n, void *stream)
{
    if (rf_status st = check_c1(ctx, "rf_c1_seed")) return st;
    if (n > ctx->capacity || (n && !items)) {
        set_error("rf_c1_seed: n %llu above capacity or NULL items", (unsigned long long)n);
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rf_device_queues q;
    rf_get_device_queues(ctx, &q);
    reserve_kernel<<<1, 32, 0, s>>>(q.outCount, n, &ctx->dev->scratch);
    RF_LAUNCHED("reserve_kernel");
    if (n) {
        seed_kernel<<<grid_for(ctx, n * 4, 8), kBlock, 0, s>>>(static_cast<const uint4 *>(items), (uint32_t)n, q,
                                                              &ctx->dev->scratch);
        RF_LAUNCHED("seed_kernel");
    }
    return RF_OK;
}

namespace rfi {
namespace {
rf_status launch_c1_work(rf_ctx *ctx, uint32_t seed, uint32_t hop, const unsigned long long *hopPtr, int32_t mode,
                         int32_t gx, int32_t gy, int32_t gz, void *retired, unsigned long long *retiredCount,
                         uint64_t retiredCapacity, int32_t deterministic, cudaStream_t s)
{
    WorkArgs a;
    rf_get_device_queues(ctx, &a.q);
    a.zipfThr = ctx->zipfThr;
    a.retired = static_cast<uint4 *>(retired);
    a.retiredCount = retiredCount;
    a.retiredCap = retiredCapacity;
    a.seed = seed;
    a.hop = hop;
    a.hopPtr = hopPtr;
    a.mode = mode;
    a.gx = gx;
    a.gy = gy;
    a.gz = gz;
    // the incoming count is only known on the device: size the grid for the
    // capacity, up to 8 resident blocks per SM, and loop
    const int grid = grid_for(ctx, (ctx->capacity + kWorkItems - 1) / kWorkItems, 8);
    time_begin(ctx, kTimeWork, s);
    if (deterministic) work_kernel<true><<<grid, kBlock, 0, s>>>(a);
    else work_kernel<false><<<grid, kBlock, 0, s>>>(a);
    RF_LAUNCHED("work_kernel");
    time_end(ctx, kTimeWork, s);
    return RF_OK;
}
}  // namespace
}  // namespace rfi

rf_status rf_c1_work(rf_ctx *ctx, uint32_t seed, uint32_t hop, int32_t mode, double zipfS, int32_t gx, int32_t gy,
                     int32_t gz, void *retired, unsigned long long *retiredCount, uint64_t retiredCapacity,
                     int32_t deterministic, void *stream)
{
    if (rf_status st = check_c1(ctx, "rf_c1_work")) return st;
    if (mode < RF_C1_UNIFORM || mode > RF_C1_NBR6 || !retired || !retiredCount) {
        set_error("rf_c1_work: bad mode or NULL retired buffer");
        return RF_ERR_ARG;
    }
    if (mode == RF_C1_NBR6 && (gx < 1 || gy < 1 || gz < 1 || gx * gy * gz != ctx->numRanks)) {
        set_error("rf_c1_work: torus %dx%dx%d does not have %d ranks", gx, gy, gz, ctx->numRanks);
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    if (mode == RF_C1_ZIPF)
        if (rf_status st = ensure_zipf(ctx, zipfS)) return st;
    return launch_c1_work(ctx, seed, hop, nullptr, mode, gx, gy, gz, retired, retiredCount, retiredCapacity,
                          deterministic, static_cast<cudaStream_t>(stream));
}

rf_status rf_c1_run(rf_ctx *ctx, const void *items, uint64_t n, uint32_t seed, int32_t mode, double zipfS,
                    int32_t gx, int32_t gy, int32_t gz, void *retired, uint64_t *retiredCountOut,
                    int32_t deterministic, int32_t hostMemory, uint32_t maxRounds, void *stream,
                    uint64_t *rounds, uint64_t *forwarded)
{
    if (rf_status st = check_c1(ctx, "rf_c1_run")) return st;
    if (n > ctx->capacity || (n && (!items || !retired)) || !retiredCountOut) {
        set_error("rf_c1_run: n %llu above capacity or NULL buffer", (unsigned long long)n);
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *devRetired = retired;
    if (hostMemory) {
        if (rf_status st = ensure_staging(ctx)) return st;
        devRetired = ctx->staging;
    }
    RF_CUDA(cudaMemsetAsync(ctx->stagingCount, 0, sizeof(unsigned long long), s));

    uint64_t active = 0, fwd = 0, r = 0;
    rf_status st;
    if (hostMemory) {
        // host items land straight in the (empty) out-queue, then get their destinations
        rf_device_queues q;
        rf_get_device_queues(ctx, &q);
        if (n) RF_CUDA(cudaMemcpyAsync(q.out, items, (size_t)n * 64u, cudaMemcpyHostToDevice, s));
        seed_dest_kernel<<<grid_for(ctx, n, 8), kBlock, 0, s>>>((uint32_t)n, q);
        RF_LAUNCHED("seed_dest_kernel");
    } else {
        st = rf_c1_seed(ctx, items, n, stream);
        if (st != RF_OK) return st;
    }
    st = rf_exchange(ctx, stream, &active);
    if (st != RF_OK) return st;
    while (active > 0) {
        if (r >= maxRounds) {
            set_error("rf_c1_run: %llu items still active after %u rounds", (unsigned long long)active, maxRounds);
            st = RF_ERR_MAX_ROUNDS;
            break;
        }
        st = rf_c1_work(ctx, seed, (uint32_t)r, mode, zipfS, gx, gy, gz, devRetired, ctx->stagingCount, n,
                        deterministic, stream);
        if (st != RF_OK) return st;
        st = rf_exchange(ctx, stream, &active);
        if (st != RF_OK) return st;
        fwd += active;
        ++r;
    }
    unsigned long long cnt = 0;
    RF_CUDA(cudaMemcpyAsync(&cnt, ctx->stagingCount, sizeof cnt, cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaStreamSynchronize(s));
    if (hostMemory && cnt)
        RF_CUDA(cudaMemcpyAsync(retired, ctx->staging, (size_t)(cnt < n ? cnt : n) * 64u, cudaMemcpyDeviceToHost, s));
    if (hostMemory) RF_CUDA(cudaStreamSynchronize(s));
    *retiredCountOut = cnt;
    if (rounds) *rounds = r;
    if (forwarded) *forwarded = fwd;
    return st == RF_ERR_MAX_ROUNDS ? st : RF_OK;
}

rf_status rf_c1_run_graph(rf_ctx *ctx, const void *items, uint64_t n, uint32_t seed, int32_t mode, double zipfS,
                          int32_t gx, int32_t gy, int32_t gz, void *retired, uint64_t *retiredCountOut,
                          int32_t deterministic, uint32_t maxRounds, void *stream, uint64_t *rounds,
                          uint64_t *forwarded)
{
    if (rf_status st = check_c1(ctx, "rf_c1_run_graph")) return st;
    if (n > ctx->capacity || (n && (!items || !retired)) || !retiredCountOut || mode < RF_C1_UNIFORM ||
        mode > RF_C1_NBR6) {
        set_error("rf_c1_run_graph: n %llu above capacity, NULL buffer or bad mode", (unsigned long long)n);
        return RF_ERR_ARG;
    }
    if (mode == RF_C1_NBR6 && (gx < 1 || gy < 1 || gz < 1 || gx * gy * gz != ctx->numRanks)) {
        set_error("rf_c1_run_graph: torus %dx%dx%d does not have %d ranks", gx, gy, gz, ctx->numRanks);
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    if (mode == RF_C1_ZIPF)
        if (rf_status st = ensure_zipf(ctx, zipfS)) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    RF_CUDA(cudaMemsetAsync(ctx->stagingCount, 0, sizeof(unsigned long long), s));
    // the loop state's first word counts finished rounds: the hop of the next
    if (!ctx->loopState) RF_CUDA(cudaMalloc(&ctx->loopState, 3 * sizeof(unsigned long long)));
    const unsigned long long *hopPtr = static_cast<const unsigned long long *>(ctx->loopState);
    uint64_t r = 0, fwd = 0;
    rf_status st = run_graph_loop(
        ctx, s, maxRounds,
        [&](cudaStream_t cs) -> rf_status {
            if (rf_status ws = launch_c1_work(ctx, seed, 0u, hopPtr, mode, gx, gy, gz, retired, ctx->stagingCount, n,
                                              deterministic, cs))
                return ws;
            return launch_exchange(ctx, cs);
        },
        &r, &fwd,
        [&](cudaStream_t cs) -> rf_status {
            if (rf_status ss = rf_c1_seed(ctx, items, n, cs)) return ss;
            return launch_exchange(ctx, cs);
        });
    if (st != RF_OK) return st;
    unsigned long long cnt = 0;
    RF_CUDA(cudaMemcpy(&cnt, ctx->stagingCount, sizeof cnt, cudaMemcpyDeviceToHost));
    *retiredCountOut = cnt;
    if (rounds) *rounds = r;
    if (forwarded) *forwarded = fwd;
    if (ctx->host->numActive) {
        set_error("rf_c1_run_graph: %llu items still active after %u rounds", (unsigned long long)ctx->host->numActive,
                  maxRounds);
        return RF_ERR_MAX_ROUNDS;
    }
    return RF_OK;
}

}  // extern "C"

namespace rfi {
int c1_shapes(int32_t *out, int32_t cap)
{
    ShapeInfo v[C1Shapes::kCount];
    C1Shapes::infos(v);
    for (int i = 0; i < C1Shapes::kCount && i < cap; ++i) {
        out[3 * i] = v[i].block;
        out[3 * i + 1] = v[i].itemsPerThread;
        out[3 * i + 2] = v[i].ctasPerSM;
    }
    return C1Shapes::kCount;
}
}  // namespace rfi

extern "C" rf_status rf_c1_run_batched(rf_ctx *ctx, const void *items, uint64_t n, uint32_t seed, int32_t mode,
                                       double zipfS, int32_t gx, int32_t gy, int32_t gz, void *retired,
                                       uint64_t *retiredCountOut, int32_t hostMemory, int32_t stepOnArrival,
                                       uint32_t maxRounds, void *stream, uint64_t *rounds, uint64_t *forwarded,
                                       unsigned long long *roundLog, uint32_t roundLogCap)
{
    using namespace rfi;
    if (rf_status st = check_c1(ctx, "rf_c1_run_batched")) return st;
    if (n > ctx->capacity || (n && (!items || !retired)) || !retiredCountOut ||
        mode < RF_C1_UNIFORM || mode > RF_C1_NBR6) {
        set_error("rf_c1_run_batched: n %llu above capacity, NULL buffer or bad mode", (unsigned long long)n);
        return RF_ERR_ARG;
    }
    if (mode == RF_C1_NBR6 && (gx < 1 || gy < 1 || gz < 1 || gx * gy * gz != ctx->numRanks)) {
        set_error("rf_c1_run_batched: torus %dx%dx%d does not have %d ranks", gx, gy, gz, ctx->numRanks);
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    if (mode == RF_C1_ZIPF)
        if (rf_status st = ensure_zipf(ctx, zipfS)) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *devRetired = retired;
    bool direct = false;
    if (hostMemory) {
        // A host buffer the device can address (page-locked memory is mapped
        // into the device's address space under unified addressing) receives
        // the retired items straight from the kernel over the host link,
        // overlapped with the rounds; any other host buffer gets them through
        // a device staging buffer and one copy after the run.
        cudaPointerAttributes pa;
        if (n && cudaPointerGetAttributes(&pa, retired) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer) {
            devRetired = pa.devicePointer;
            direct = true;
        } else {
            (void)cudaGetLastError();
            if (rf_status st = ensure_staging(ctx)) return st;
            devRetired = ctx->staging;
        }
    }
    RF_CUDA(cudaMemsetAsync(ctx->stagingCount, 0, sizeof(unsigned long long), s));
    rf_device_queues q;
    rf_get_device_queues(ctx, &q);
    // With steps on arrival the kernel's first scatter reads 16-byte aligned
    // device items where the caller keeps them; only their first ranks are
    // written.  Otherwise the items are copied into the out-queue first.
    const bool inPlace = !hostMemory && stepOnArrival && ((uintptr_t)items & 15u) == 0;
    if (hostMemory) {
        if (n) RF_CUDA(cudaMemcpyAsync(q.out, items, (size_t)n * 64u, cudaMemcpyHostToDevice, s));
        seed_dest_kernel<<<grid_for(ctx, n, 8), kBlock, 0, s>>>((uint32_t)n, q);
        RF_LAUNCHED("seed_dest_kernel");
    } else if (inPlace) {
        seed_dest_kernel<<<grid_for(ctx, n, 8), kBlock, 0, s>>>((uint32_t)n, q);
        RF_LAUNCHED("seed_dest_kernel");
    } else {
        if (rf_status st = rf_c1_seed(ctx, items, n, stream)) return st;
    }
    // with steps on arrival the persistent kernel delivers the seeded
    // out-queue itself (a pre-round that applies round 0's step on arrival);
    // otherwise the seed exchange runs first, asynchronously
    if (!stepOnArrival)
        if (rf_status st = rf_exchange(ctx, stream, nullptr)) return st;

    C1Work w;
    w.zipfThr = ctx->zipfThr;
    w.seed = seed;
    w.mode = mode;
    w.gx = gx;
    w.gy = gy;
    w.gz = gz;
    w.R = ctx->numRanks;
    unsigned long long res[4];
    rf_status st = C1Shapes::launch(ctx->batchedShape[RF_POLICY_MICROBENCH], ctx, w, maxRounds, s, roundLog,
                                    roundLogCap, static_cast<uint4 *>(devRetired), n,
                                 ctx->stagingCount, res, stepOnArrival != 0, stepOnArrival != 0,
                                 inPlace ? items : nullptr);
    if (st != RF_OK) return st;
    unsigned long long cnt = 0;
    RF_CUDA(cudaMemcpy(&cnt, ctx->stagingCount, sizeof cnt, cudaMemcpyDeviceToHost));
    if (hostMemory && !direct && cnt)
        RF_CUDA(cudaMemcpyAsync(retired, ctx->staging, (size_t)(cnt < n ? cnt : n) * 64u, cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaStreamSynchronize(s));
    *retiredCountOut = cnt;
    if (rounds) *rounds = res[0];
    if (forwarded) *forwarded = res[1];
    if (ctx->host->numActive) {
        set_error("rf_c1_run_batched: %llu items still active after %u rounds",
                  (unsigned long long)ctx->host->numActive, maxRounds);
        return RF_ERR_MAX_ROUNDS;
    }
    return RF_OK;
}

// Several runs from page-locked host memory: one persistent launch per run,
// pipelined over the two directions of the host link.  While run k's kernel
// executes, run k + 1's items are copied in on the context's copy stream,
// and run k's retired items are copied out on its copy-out stream as soon
// as their sink slots are final (the kernel publishes that count in mapped
// host memory after every round; the host copies it out in chunks of at
// least 2^20 items while it waits for the launch).  The
// items of run k are staged in the queue slots [n, 2n) of `in` (k even) or of
// `out` (k odd), beyond the [0, n) a run's kernel uses, and read there in
// place; run k retires into the staging buffer's slots [k n, (k + 1) n).
// Each launch is rf_c1_run_batched's, so each run's results are those of its
// own launch.
static rf_status c1_runs_pipelined(rf_ctx *ctx, const void *items, uint64_t n, int32_t numRuns, uint32_t seed,
                                   const int32_t *modes, int32_t gx, int32_t gy, int32_t gz, void *hostRetired,
                                   uint64_t *retiredCountsOut, uint32_t maxRounds, cudaStream_t s,
                                   uint64_t *roundsOut, uint64_t *forwarded, const rf_device_queues &q)
{
    using namespace rfi;
    if (rf_status st = ensure_copy_stream(ctx)) return st;
    if (rf_status st = ensure_staging(ctx)) return st;
    uint4 *sink = static_cast<uint4 *>(ctx->staging);
    cudaStream_t cs = ctx->copyStream, co = ctx->copyOutStream;
    const size_t runBytes = (size_t)n * 64u;
    void *slot[2] = {static_cast<unsigned char *>(q.in) + runBytes, static_cast<unsigned char *>(q.out) + runBytes};
    // the first copy waits for whatever the caller's stream still has in flight
    RF_CUDA(cudaEventRecord(ctx->copyDone[1], s));
    RF_CUDA(cudaStreamWaitEvent(cs, ctx->copyDone[1], 0));
    RF_CUDA(cudaMemcpyAsync(slot[0], items, runBytes, cudaMemcpyHostToDevice, cs));
    RF_CUDA(cudaEventRecord(ctx->copyDone[0], cs));
    unsigned long long fwd = 0;
    rf_status st = RF_OK;
    for (int32_t k = 0; k < numRuns && st == RF_OK; ++k) {
        const int b = k & 1;
        // slot b ^ 1 was last read by run k - 1, whose launch has completed
        if (k + 1 < numRuns) {
            RF_CUDA(cudaMemcpyAsync(slot[b ^ 1], static_cast<const unsigned char *>(items) + (size_t)(k + 1) * runBytes,
                                    runBytes, cudaMemcpyHostToDevice, cs));
            RF_CUDA(cudaEventRecord(ctx->copyDone[b ^ 1], cs));
        }
        RF_CUDA(cudaStreamWaitEvent(s, ctx->copyDone[b], 0));
        seed_dest_kernel<<<grid_for(ctx, n, 8), kBlock, 0, s>>>((uint32_t)n, q);
        RF_LAUNCHED("seed_dest_kernel");
        C1Work w;
        w.zipfThr = ctx->zipfThr;
        w.seed = seed;
        w.mode = modes[k];
        w.gx = gx;
        w.gy = gy;
        w.gz = gz;
        w.R = ctx->numRanks;
        unsigned long long res[4];
        volatile unsigned long long *prog = ctx->progressHost;
        *prog = 0ull;
        unsigned long long copied = 0;  // retired items of run k already on their way out
        unsigned char *hostRun = static_cast<unsigned char *>(hostRetired) + (size_t)k * runBytes;
        const uint4 *sinkRun = sink + (size_t)k * n * 4u;
        cudaError_t copyErr = cudaSuccess;
        const std::function<void()> poll = [&]() {
            const unsigned long long p = *prog;  // final sink slots so far (never more than n)
            if (p >= copied + (1ull << 20) && p <= n && copyErr == cudaSuccess) {
                copyErr = cudaMemcpyAsync(hostRun + (size_t)copied * 64u, sinkRun + (size_t)copied * 4u,
                                          (size_t)(p - copied) * 64u, cudaMemcpyDeviceToHost, co);
                copied = p;
            } else {
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        };
        st = C1ProgressShapes::launch(ctx->batchedShape[RF_POLICY_MICROBENCH], ctx, C1WorkProgress(w), maxRounds, s,
                                      nullptr, 0u, sink + (size_t)k * n * 4u, (unsigned long long)n,
                                      ctx->stagingCount, res, true, true, slot[b], 1u, 0ull, nullptr,
                                      ctx->progressDev, &poll);
        if (copyErr != cudaSuccess) {
            cuda_fail(copyErr, "cudaMemcpyAsync of retired items");
            st = RF_ERR_CUDA;
        }
        if (st != RF_OK) break;
        // the launch has completed: the rest of its retired items go out while the next run executes
        const unsigned long long got = res[3] < n ? res[3] : n;
        if (got > copied)
            RF_CUDA(cudaMemcpyAsync(hostRun + (size_t)copied * 64u, sinkRun + (size_t)copied * 4u,
                                    (size_t)(got - copied) * 64u, cudaMemcpyDeviceToHost, co));
        retiredCountsOut[k] = res[3];
        if (roundsOut) roundsOut[k] = res[0];
        fwd += res[1];
        if (ctx->host->numActive) {
            set_error("rf_c1_run_batched_runs: run %d: %llu items still active after %u rounds", k,
                      (unsigned long long)ctx->host->numActive, maxRounds);
            st = RF_ERR_MAX_ROUNDS;
        }
    }
    // no copy may still be writing into the queues or the host buffer when the call returns
    RF_CUDA(cudaStreamSynchronize(cs));
    RF_CUDA(cudaStreamSynchronize(co));
    if (forwarded) *forwarded = fwd;
    return st;
}

// Several independent runs of the microbenchmark in one persistent launch.
// Run k holds items [k n, (k + 1) n) of `items`, all of them starting at rank
// i mod R as in a run of its own, and moves under its own destination law
// modes[k]; its retired items land, in its own order, in retired slots
// [k n, (k + 1) n).  The runs share the ranks' queues: a round's queue of
// rank r holds the items of every run bound for r, and a stable partition of
// the whole queue, restricted to one run, is that run's own stable partition,
// so every run's queues and retirements equal those of its own launch.
extern "C" rf_status rf_c1_run_batched_runs(rf_ctx *ctx, const void *items, uint64_t n, int32_t numRuns,
                                            uint32_t seed, const int32_t *modes, double zipfS, int32_t gx,
                                            int32_t gy, int32_t gz, void *retired, uint64_t *retiredCountsOut,
                                            int32_t hostMemory, uint32_t maxRounds, void *stream,
                                            uint64_t *roundsOut, uint64_t *forwarded, unsigned long long *roundLog,
                                            uint32_t roundLogCap)
{
    using namespace rfi;
    if (rf_status st = check_c1(ctx, "rf_c1_run_batched_runs")) return st;
    if (numRuns < 1 || numRuns > kMaxRuns || !modes || !retiredCountsOut) {
        set_error("rf_c1_run_batched_runs: %d runs (1 to %d) or a NULL mode / count array", numRuns, kMaxRuns);
        return RF_ERR_ARG;
    }
    const unsigned long long total = (unsigned long long)numRuns * n;
    if (total > ctx->capacity || total >= (1ull << 31) || (n && (!items || !retired))) {
        set_error("rf_c1_run_batched_runs: %d x %llu items above capacity %llu or 2^31, or a NULL buffer", numRuns,
                  (unsigned long long)n, (unsigned long long)ctx->capacity);
        return RF_ERR_ARG;
    }
    bool anyZipf = false, anyTorus = false;
    uint32_t laws = 0;
    for (int32_t k = 0; k < numRuns; ++k) {
        if (modes[k] < RF_C1_UNIFORM || modes[k] > RF_C1_NBR6) {
            set_error("rf_c1_run_batched_runs: run %d has bad mode %d", k, modes[k]);
            return RF_ERR_ARG;
        }
        laws |= (uint32_t)modes[k] << (2 * k);
        anyZipf |= modes[k] == RF_C1_ZIPF;
        anyTorus |= modes[k] == RF_C1_NBR6;
    }
    if (anyTorus && (gx < 1 || gy < 1 || gz < 1 || gx * gy * gz != ctx->numRanks)) {
        set_error("rf_c1_run_batched_runs: torus %dx%dx%d does not have %d ranks", gx, gy, gz, ctx->numRanks);
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    if (anyZipf)
        if (rf_status st = ensure_zipf(ctx, zipfS)) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *devRetired = retired;
    bool direct = false;
    if (hostMemory) {
        // as rf_c1_run_batched: page-locked host memory receives the retired
        // items from the kernel, any other host buffer through a staging copy
        cudaPointerAttributes pa;
        if (n && cudaPointerGetAttributes(&pa, retired) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer) {
            devRetired = pa.devicePointer;
            direct = true;
        } else {
            (void)cudaGetLastError();
            if (rf_status st = ensure_staging(ctx)) return st;
            devRetired = ctx->staging;
        }
    }
    RF_CUDA(cudaMemsetAsync(ctx->stagingCount, 0, sizeof(unsigned long long), s));
    rf_device_queues q;
    rf_get_device_queues(ctx, &q);
    if (direct && numRuns > 1)
        return c1_runs_pipelined(ctx, items, n, numRuns, seed, modes, gx, gy, gz, retired, retiredCountsOut,
                                 maxRounds, s, roundsOut, forwarded, q);
    // the seeded items are read where the caller keeps them when they are
    // 16-byte aligned device memory, else copied into the out-queue first
    const bool inPlace = !hostMemory && ((uintptr_t)items & 15u) == 0;
    if (total && !inPlace)
        RF_CUDA(cudaMemcpyAsync(q.out, items, (size_t)total * 64u,
                                hostMemory ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    seed_dest_runs_kernel<<<grid_for(ctx, total, 8), kBlock, 0, s>>>((uint32_t)total, n ? (uint32_t)n : 1u, q);
    RF_LAUNCHED("seed_dest_runs_kernel");

    C1Work w;
    w.zipfThr = ctx->zipfThr;
    w.seed = seed;
    w.mode = modes[0];
    w.gx = gx;
    w.gy = gy;
    w.gz = gz;
    w.R = ctx->numRanks;
    w.runs = numRuns;
    w.laws = laws;
    auto lg2 = [](int32_t v) { return (v > 0 && (v & (v - 1)) == 0) ? __builtin_ctz((unsigned)v) : -1; };
    if (anyTorus && lg2(gx) >= 0 && lg2(gy) >= 0 && lg2(gz) >= 0) {
        w.lgx = lg2(gx);
        w.lgy = lg2(gy);
    }
    unsigned long long res[4], runRes[2 * kMaxRuns];
    rf_status st = C1Shapes::launch(ctx->batchedShape[RF_POLICY_MICROBENCH], ctx, w, maxRounds, s, roundLog,
                                    roundLogCap, static_cast<uint4 *>(devRetired), total, ctx->stagingCount, res,
                                    true, true, inPlace ? items : nullptr, (uint32_t)numRuns,
                                    (unsigned long long)n, runRes);
    if (st != RF_OK) return st;
    if (hostMemory && !direct && total)
        RF_CUDA(cudaMemcpyAsync(retired, ctx->staging, (size_t)total * 64u, cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaStreamSynchronize(s));
    for (int32_t k = 0; k < numRuns; ++k) {
        retiredCountsOut[k] = runRes[kMaxRuns + k];
        if (roundsOut) roundsOut[k] = runRes[k];
    }
    if (forwarded) *forwarded = res[1];
    if (ctx->host->numActive) {
        set_error("rf_c1_run_batched_runs: %llu items still active after %u rounds",
                  (unsigned long long)ctx->host->numActive, maxRounds);
        return RF_ERR_MAX_ROUNDS;
    }
    return RF_OK;
}
