// forwardRays() on one device (Sec. 4.2): the exchange that moves every
// emitted item to its destination rank's incoming segment.
//
// The paper sorts 64-bit keys (dest << 32 | i) with a radix sort, gathers the
// items in key order (Sec. 4.2.1), finds each rank's begin/end, and ships the
// blocks with MPI_Alltoall(v) (Sec. 4.2.2); the result on every rank is the
// stable partition of the emitted items by destination.  With all ranks in
// one HBM the same result is a single-digit stable counting sort, and the
// delivery is the scatter itself:
//
//   count    per tile of the out-queue, a histogram of destinations (warp
//            aggregated with __match_any_sync), written digit-major, plus the
//            per-destination totals;
//   scan     one CTA per destination: the destination's global offset (sum of
//            the totals before it) plus the exclusive scan of its per-tile
//            counts = where each tile's items for that destination go; CTA 0
//            also writes the per-rank segment offsets and the total
//            (Sec. 4.2.3's reduce-add of received counts);
//   scatter  per tile: a bulk asynchronous copy stages the tile's items in
//            shared memory while the warps rank every item within its
//            destination (match_any + popc, per-warp counters, scan over
//            warps); the items are then written out grouped by destination,
//            so consecutive threads store consecutive 16-byte vectors;
//   wrap-up  clears the append counter and per-exchange accumulators and
//            records the exchange's statistics (Sec. 4.2.3).
//
// All kernels read the item count from the device-side append counter, so a
// round needs no host round trip; grids are sized to the SM count and loop
// over tiles.
#include <cstring>

#include "internal.cuh"

namespace rfi {

namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;

struct ExArgs {
    const void *out;
    const int32_t *dest;
    void *in;
    uint32_t *inOffset;
    uint32_t *count;
    uint32_t *tileHist;
    DevState *state;
    uint64_t capacity;
    uint32_t tileItems;
    uint32_t maxTiles;
    uint32_t itemBytes;
    int32_t numRanks;
};

__device__ __forceinline__ uint32_t items_in_queue(const ExArgs &a)
{
    unsigned long long c = a.state->outCount;
    return (uint32_t)(c < a.capacity ? c : a.capacity);
}

// Exclusive scan of v[0..n) in shared memory (n <= 4 * kBlock), in place, by
// the whole block.  Returns the total.  Contains __syncthreads at entry/exit.
__device__ uint32_t block_exclusive_scan(uint32_t *v, int n, uint32_t *tmp)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __syncthreads();
    uint32_t x[4];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int i = tid * 4 + j;
        x[j] = i < n ? v[i] : 0u;
        uint32_t t = x[j];
        x[j] = sum;
        sum += t;
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kWarps ? tmp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kWarps) tmp[lane] = wi - w;
        if (lane == 31) tmp[kWarps] = wi;
    }
    __syncthreads();
    const uint32_t base = tmp[warp] + incl - sum;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int i = tid * 4 + j;
        if (i < n) v[i] = base + x[j];
    }
    const uint32_t total = tmp[kWarps];
    __syncthreads();
    return total;
}

// ---------------------------------------------------------------------------
// count: per-tile destination histograms (digit-major) and per-destination totals
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) count_kernel(ExArgs a)
{
    extern __shared__ uint32_t hist[];
    const int R = a.numRanks;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t n = items_in_queue(a);
    const uint32_t numTiles = (n + a.tileItems - 1) / a.tileItems;
    uint32_t acc[RF_MAX_RANKS / kBlock] = {};
    unsigned long long bad = 0, holes = 0;
    for (uint32_t t = blockIdx.x; t < numTiles; t += gridDim.x) {
        for (int e = tid; e < R; e += kBlock) hist[e] = 0;
        __syncthreads();
        const uint32_t begin = t * a.tileItems;
        const uint32_t cnt = min(a.tileItems, n - begin);
        for (uint32_t b = 0; b < cnt; b += kBlock) {
            const uint32_t i = b + tid;
            const int32_t d = i < cnt ? __ldg(a.dest + begin + i) : -1;
            const bool valid = (uint32_t)d < (uint32_t)R;
            const int key = valid ? d : R;
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
            if (valid) {
                if (lane == __ffs(peers) - 1) atomicAdd(&hist[d], (uint32_t)__popc(peers));
            } else if (i < cnt) {
                if (d == -1) holes++;
                else bad++;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < RF_MAX_RANKS / kBlock; ++j) {
            const int e = tid + j * kBlock;
            if (e < R) {
                const uint32_t c = hist[e];
                a.tileHist[(size_t)e * a.maxTiles + t] = c;
                acc[j] += c;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < RF_MAX_RANKS / kBlock; ++j) {
        const int e = tid + j * kBlock;
        if (e < R && acc[j]) atomicAdd(&a.count[e], acc[j]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bad += __shfl_down_sync(0xFFFFFFFFu, bad, o);
        holes += __shfl_down_sync(0xFFFFFFFFu, holes, o);
    }
    if (lane == 0) {
        if (bad) atomicAdd(&a.state->bad, bad);
        if (holes) atomicAdd(&a.state->holes, holes);
    }
}

// ---------------------------------------------------------------------------
// scan: CTA d turns row d of tileHist into absolute output positions
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) scan_kernel(ExArgs a)
{
    __shared__ uint32_t tmp[kWarps + 1];
    __shared__ uint32_t vals[4 * kBlock];
    __shared__ uint32_t red[kWarps];
    const int R = a.numRanks;
    const int d = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = items_in_queue(a);
    const uint32_t numTiles = (n + a.tileItems - 1) / a.tileItems;

    // global offset of destination d: sum of the totals before it
    uint32_t part = 0;
    for (int e = tid; e < d; e += kBlock) part += a.count[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xFFFFFFFFu, part, o);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    uint32_t offD = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) offD += red[w];

    if (d == 0) {
        // per-rank segment offsets and the total
        for (int c = 0; c < R; c += 4 * kBlock) {
            const int m = min(4 * kBlock, R - c);
            for (int e = tid; e < m; e += kBlock) vals[e] = a.count[c + e];
            const uint32_t carry = c ? a.inOffset[c] : 0u;  // written by this CTA in the previous chunk
            const uint32_t tot = block_exclusive_scan(vals, m, tmp);
            for (int e = tid; e < m; e += kBlock) a.inOffset[c + e] = carry + vals[e];
            if (tid == 0) a.inOffset[c + m] = carry + tot;
            __syncthreads();
        }
        if (tid == 0) a.state->numActive = a.inOffset[R];
    }

    uint32_t *row = a.tileHist + (size_t)d * a.maxTiles;
    uint32_t running = offD;
    for (uint32_t c = 0; c < numTiles; c += 4 * kBlock) {
        const int m = (int)min((uint32_t)(4 * kBlock), numTiles - c);
        for (int e = tid; e < m; e += kBlock) vals[e] = row[c + e];
        const uint32_t tot = block_exclusive_scan(vals, m, tmp);
        for (int e = tid; e < m; e += kBlock) row[c + e] = running + vals[e];
        running += tot;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// scatter: stage a tile in shared memory, rank within destination, write out
// grouped by destination.  V = 16-byte vectors per item (0: runtime), K =
// items per thread per tile (tile = 256 K items).
// ---------------------------------------------------------------------------
struct ScatterLayout {
    uint32_t items, wc, cnt, start, base, slotSrc, slotDst, tmp, bar, total;
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline ScatterLayout scatter_layout(uint32_t tileItems, uint32_t itemBytes, int R)
{
    ScatterLayout L;
    uint32_t o = 0;
    L.items = o;   o = align_up(o + tileItems * itemBytes, 128);
    L.wc = o;      o = align_up(o + kWarps * R * 4u, 16);
    L.cnt = o;     o = align_up(o + R * 4u, 16);
    L.start = o;   o = align_up(o + R * 4u, 16);
    L.base = o;    o = align_up(o + R * 4u, 16);
    L.slotSrc = o; o = align_up(o + tileItems * 2u, 16);
    L.slotDst = o; o = align_up(o + tileItems * 4u, 16);
    L.tmp = o;     o = align_up(o + (kWarps + 1) * 4u, 16);
    L.bar = o;     o = align_up(o + 8u, 16);
    L.total = o;
    return L;
}

template <int V, int K>
__global__ void __launch_bounds__(kBlock) scatter_kernel(ExArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int R = a.numRanks;
    const ScatterLayout L = scatter_layout(a.tileItems, a.itemBytes, R);
    uint4 *sItems = reinterpret_cast<uint4 *>(smem + L.items);
    uint32_t *wc = reinterpret_cast<uint32_t *>(smem + L.wc);
    uint32_t *dCnt = reinterpret_cast<uint32_t *>(smem + L.cnt);
    uint32_t *dStart = reinterpret_cast<uint32_t *>(smem + L.start);
    uint32_t *dBase = reinterpret_cast<uint32_t *>(smem + L.base);
    uint16_t *slotSrc = reinterpret_cast<uint16_t *>(smem + L.slotSrc);
    uint32_t *slotDst = reinterpret_cast<uint32_t *>(smem + L.slotDst);
    uint32_t *tmp = reinterpret_cast<uint32_t *>(smem + L.tmp);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t vpi = V ? (uint32_t)V : a.itemBytes / 16u;  // vectors per item
    const uint32_t n = items_in_queue(a);
    const uint32_t numTiles = (n + a.tileItems - 1) / a.tileItems;
    if (blockIdx.x >= numTiles) return;

    if (tid == 0) {
        mbar_init(bar, 1);
        fence_proxy_async_smem();
    }
    __syncthreads();

    uint32_t phase = 0;
    for (uint32_t t = blockIdx.x; t < numTiles; t += gridDim.x) {
        const uint32_t begin = t * a.tileItems;
        const uint32_t cnt = min(a.tileItems, n - begin);
        if (tid == 0) {
            // the previous tile's generic-proxy reads of sItems are ordered
            // before this async-proxy write by the barrier that ended it
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, cnt * a.itemBytes);
            bulk_g2s(sItems, static_cast<const unsigned char *>(a.out) + (size_t)begin * a.itemBytes,
                     cnt * a.itemBytes, bar);
        }
        for (int e = lane; e < R; e += 32) wc[warp * R + e] = 0u;
        __syncwarp();

        // rank every item within its destination, per warp, in index order
        int myD[K];
        uint32_t myR[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint32_t idx = (uint32_t)(warp * 32 * K + k * 32 + lane);
            const int32_t d = idx < cnt ? __ldg(a.dest + begin + idx) : -1;
            const bool valid = (uint32_t)d < (uint32_t)R;
            const int key = valid ? d : R;
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
            const int leader = __ffs(peers) - 1;
            uint32_t old = 0;
            if (valid && lane == leader) {
                old = wc[warp * R + d];
                wc[warp * R + d] = old + (uint32_t)__popc(peers);
            }
            old = __shfl_sync(0xFFFFFFFFu, old, leader);
            __syncwarp();
            myD[k] = valid ? d : -1;
            myR[k] = old + (uint32_t)__popc(peers & lanemask_lt());
        }
        __syncthreads();

        // per destination: exclusive scan over warps, tile count, tile base
        for (int e = tid; e < R; e += kBlock) {
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = wc[w * R + e];
                wc[w * R + e] = s;
                s += c;
            }
            dCnt[e] = s;
            dStart[e] = s;
            dBase[e] = s ? a.tileHist[(size_t)e * a.maxTiles + t] : 0u;
        }
        const uint32_t nValid = block_exclusive_scan(dStart, R, tmp);

        // slot of each item in the destination-grouped tile, and its final position
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (myD[k] >= 0) {
                const int d = myD[k];
                const uint32_t within = wc[warp * R + d] + myR[k];
                const uint32_t slot = dStart[d] + within;
                slotSrc[slot] = (uint16_t)(warp * 32 * K + k * 32 + lane);
                slotDst[slot] = dBase[d] + within;
            }
        }

        const bool ok = mbar_wait_bounded(bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(&a.state->status, RF_DEV_TIMEOUT);
                (void)mbar_wait_bounded(bar, phase ^ 1u);  // let the copy in flight land
            }
            return;
        }

        // write out: consecutive threads, consecutive 16-byte vectors of the
        // destination-grouped tile
        uint4 *dq = static_cast<uint4 *>(a.in);
        const uint32_t total = nValid * vpi;
        for (uint32_t v = tid; v < total; v += kBlock) {
            const uint32_t slot = v / vpi;
            const uint32_t part = v - slot * vpi;
            dq[(size_t)slotDst[slot] * vpi + part] = sItems[(uint32_t)slotSrc[slot] * vpi + part];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// wrap-up (Sec. 4.2.3)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) wrapup_kernel(ExArgs a)
{
    for (int e = threadIdx.x; e < a.numRanks; e += kBlock) a.count[e] = 0u;
    if (threadIdx.x == 0) {
        DevState *s = a.state;
        const unsigned long long oc = s->outCount;
        const unsigned long long emitted = oc < a.capacity ? oc : a.capacity;
        s->lastEmitted = emitted;
        s->lastDropped = oc - emitted;
        s->lastBad = s->bad;
        s->lastHoles = s->holes;
        s->exchanges += 1ull;
        s->totalDelivered += s->numActive;
        s->totalDropped += (oc - emitted) + s->bad;
        s->outCount = 0ull;
        s->bad = 0ull;
        s->holes = 0ull;
    }
}

using ExKernel = void (*)(ExArgs);

struct ScatterChoice {
    ExKernel fn;
    uint32_t k;
};

// The scatter variants built for an item size (K = items per thread, tile =
// 256 K items), largest tile first; the first is the default.  A tile stays
// within 64 KiB of shared memory.
constexpr int kMaxVariants = 3;

int scatter_variants(uint32_t itemBytes, ScatterChoice out[kMaxVariants])
{
    switch (itemBytes / 16u) {
    case 1:
        out[0] = {scatter_kernel<1, 16>, 16};
        out[1] = {scatter_kernel<1, 8>, 8};
        out[2] = {scatter_kernel<1, 4>, 4};
        return 3;
    case 2:
        out[0] = {scatter_kernel<2, 8>, 8};
        out[1] = {scatter_kernel<2, 4>, 4};
        out[2] = {scatter_kernel<2, 2>, 2};
        return 3;
    case 3:
        out[0] = {scatter_kernel<3, 4>, 4};
        out[1] = {scatter_kernel<3, 2>, 2};
        out[2] = {scatter_kernel<3, 1>, 1};
        return 3;
    case 4:
        out[0] = {scatter_kernel<4, 4>, 4};
        out[1] = {scatter_kernel<4, 2>, 2};
        out[2] = {scatter_kernel<4, 1>, 1};
        return 3;
    case 8:
        out[0] = {scatter_kernel<8, 2>, 2};
        out[1] = {scatter_kernel<8, 1>, 1};
        return 2;
    default:
        break;
    }
    int m = 0;
    if (256u * 4u * itemBytes <= 65536u) out[m++] = {scatter_kernel<0, 4>, 4};
    if (256u * 2u * itemBytes <= 65536u) out[m++] = {scatter_kernel<0, 2>, 2};
    out[m++] = {scatter_kernel<0, 1>, 1};
    return m;
}

// The variant with K items per thread (k = 0: the default); {nullptr, 0} if none.
ScatterChoice pick_scatter(uint32_t itemBytes, uint32_t k = 0)
{
    ScatterChoice v[kMaxVariants];
    const int m = scatter_variants(itemBytes, v);
    if (k == 0) return v[0];
    for (int i = 0; i < m; ++i)
        if (v[i].k == k) return v[i];
    return {nullptr, 0u};
}

ExArgs make_args(rf_ctx *ctx)
{
    ExArgs a;
    a.out = ctx->out;
    a.dest = ctx->dest;
    a.in = ctx->in;
    a.inOffset = ctx->inOffset;
    a.count = ctx->count;
    a.tileHist = ctx->tileHist;
    a.state = ctx->dev;
    a.capacity = ctx->capacity;
    a.tileItems = ctx->tileItems;
    a.maxTiles = ctx->maxTiles;
    a.itemBytes = ctx->itemBytes;
    a.numRanks = ctx->numRanks;
    return a;
}

}  // namespace

// Chooses the tile size and grid shapes for a context (called by rf_create /
// rf_resize and when a configuration is set): the requested ones where the
// context holds a request, else the defaults.
rf_status configure_exchange(rf_ctx *ctx)
{
    ScatterChoice c = pick_scatter(ctx->itemBytes, ctx->reqScatterK);
    if (!c.fn) {
        set_error("no scatter variant with %u items per thread for %u-byte items", ctx->reqScatterK, ctx->itemBytes);
        return RF_ERR_ARG;
    }
    ctx->tileItems = 256u * c.k;
    const uint64_t tiles = (ctx->capacity + ctx->tileItems - 1) / ctx->tileItems;
    ctx->maxTiles = (uint32_t)((tiles + 3) / 4 * 4);
    ctx->scatterSmem = scatter_layout(ctx->tileItems, ctx->itemBytes, ctx->numRanks).total;
    // the attribute is per kernel, shared by every context: allow the device
    // maximum once so no context lowers it below another's need
    int optin = 0;
    RF_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    if ((int)ctx->scatterSmem > optin) {
        set_error("scatter tile needs %zu bytes of shared memory, the device allows %d", ctx->scatterSmem, optin);
        return RF_ERR_ARG;
    }
    RF_CUDA(cudaFuncSetAttribute(c.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    int perSM = 0;
    RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perSM, c.fn, kBlock, ctx->scatterSmem));
    if (perSM < 1) {
        set_error("scatter kernel does not fit on an SM (%zu bytes of shared memory)", ctx->scatterSmem);
        return RF_ERR_ARG;
    }
    ctx->scatterBlocks = ctx->reqScatterBlocks > 0 ? ctx->reqScatterBlocks : ctx->numSMs * perSM;
    int cperSM = 0;
    RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cperSM, count_kernel, kBlock,
                                                          (size_t)ctx->numRanks * 4u));
    ctx->countBlocks = ctx->reqCountBlocks > 0 ? ctx->reqCountBlocks : ctx->numSMs * (cperSM < 1 ? 1 : cperSM);
    return RF_OK;
}

// Per-tile histograms for the configured tile: grown (never shrunk) when a
// smaller tile needs more of them.  Waits for the device before freeing.
rf_status ensure_tile_hist(rf_ctx *ctx)
{
    if (ctx->tileHist && ctx->tileHistTiles >= ctx->maxTiles) return RF_OK;
    RF_CUDA(cudaDeviceSynchronize());
    cudaFree(ctx->tileHist);
    ctx->tileHist = nullptr;
    ctx->tileHistTiles = 0;
    RF_CUDA(cudaMalloc(&ctx->tileHist, (size_t)ctx->numRanks * ctx->maxTiles * sizeof(uint32_t)));
    ctx->tileHistTiles = ctx->maxTiles;
    return RF_OK;
}

// count, scan and scatter of the out-queue into the incoming queue (no wrap-up)
rf_status launch_partition(rf_ctx *ctx, cudaStream_t s)
{
    const ExArgs a = make_args(ctx);
    const ScatterChoice c = pick_scatter(ctx->itemBytes, ctx->tileItems / 256u);
    const int maxTiles = (int)ctx->maxTiles;
    const int cb = ctx->countBlocks < maxTiles ? ctx->countBlocks : maxTiles;
    const int sb = ctx->scatterBlocks < maxTiles ? ctx->scatterBlocks : maxTiles;

    time_begin(ctx, kTimeCount, s);
    count_kernel<<<cb, kBlock, (size_t)ctx->numRanks * 4u, s>>>(a);
    RF_LAUNCHED("count_kernel");
    time_end(ctx, kTimeCount, s);

    time_begin(ctx, kTimeScan, s);
    scan_kernel<<<ctx->numRanks, kBlock, 0, s>>>(a);
    RF_LAUNCHED("scan_kernel");
    time_end(ctx, kTimeScan, s);

    time_begin(ctx, kTimeScatter, s);
    c.fn<<<sb, kBlock, ctx->scatterSmem, s>>>(a);
    RF_LAUNCHED("scatter_kernel");
    time_end(ctx, kTimeScatter, s);
    return RF_OK;
}

rf_status launch_exchange(rf_ctx *ctx, cudaStream_t s)
{
    if (rf_status st = launch_partition(ctx, s)) return st;
    const ExArgs a = make_args(ctx);
    wrapup_kernel<<<1, kBlock, 0, s>>>(a);
    RF_LAUNCHED("wrapup_kernel");
    return RF_OK;
}

}  // namespace rfi

extern "C" rf_status rf_exchange(rf_ctx *ctx, void *stream, uint64_t *numActiveOut)
{
    if (!ctx) {
        rfi::set_error("rf_exchange: NULL context");
        return RF_ERR_ARG;
    }
    rfi::DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rf_status st = rfi::launch_exchange(ctx, s);
    if (st != RF_OK) return st;
    RF_CUDA(cudaMemcpyAsync(ctx->host, ctx->dev, sizeof(rfi::DevState), cudaMemcpyDeviceToHost, s));
    ctx->lastStream = s;
    ctx->pending = true;
    if (!numActiveOut) return RF_OK;
    st = rfi::sync_state(ctx);
    *numActiveOut = ctx->host->numActive;
    return st;
}

// ---------------------------------------------------------------------------
// Exchange configuration and its autotuner: tile size (items per scatter
// tile) and the grid sizes of the count and scatter kernels.
// ---------------------------------------------------------------------------
namespace {

rf_status apply_config(rf_ctx *ctx, uint32_t k, int scatterBlocks, int countBlocks)
{
    const uint32_t oldK = ctx->reqScatterK;
    const int oldS = ctx->reqScatterBlocks, oldC = ctx->reqCountBlocks;
    ctx->reqScatterK = k;
    ctx->reqScatterBlocks = scatterBlocks;
    ctx->reqCountBlocks = countBlocks;
    rf_status st = rfi::configure_exchange(ctx);
    if (st == RF_OK) st = rfi::ensure_tile_hist(ctx);
    if (st != RF_OK) {
        ctx->reqScatterK = oldK;
        ctx->reqScatterBlocks = oldS;
        ctx->reqCountBlocks = oldC;
        (void)rfi::configure_exchange(ctx);
    }
    return st;
}

}  // namespace

extern "C" rf_status rf_get_exchange_config(rf_ctx *ctx, rf_exchange_config *out)
{
    if (!ctx || !out) {
        rfi::set_error("rf_get_exchange_config: NULL argument");
        return RF_ERR_ARG;
    }
    out->tileItems = ctx->tileItems;
    out->scatterBlocks = ctx->scatterBlocks;
    out->countBlocks = ctx->countBlocks;
    return RF_OK;
}

extern "C" rf_status rf_set_exchange_config(rf_ctx *ctx, const rf_exchange_config *cfg)
{
    using namespace rfi;
    if (!ctx || !cfg) {
        set_error("rf_set_exchange_config: NULL argument");
        return RF_ERR_ARG;
    }
    if (cfg->tileItems % 256u || cfg->scatterBlocks < 0 || cfg->countBlocks < 0 || cfg->scatterBlocks > (1 << 20) ||
        cfg->countBlocks > (1 << 20) ||
        (cfg->tileItems && !pick_scatter(ctx->itemBytes, cfg->tileItems / 256u).fn)) {
        set_error("rf_set_exchange_config: tile of %u items, grids %d / %d not available for %u-byte items",
                  cfg->tileItems, cfg->scatterBlocks, cfg->countBlocks, ctx->itemBytes);
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    return apply_config(ctx, cfg->tileItems / 256u, cfg->scatterBlocks, cfg->countBlocks);
}

extern "C" rf_status rf_tune_exchange(rf_ctx *ctx, void *stream, uint32_t trials, rf_exchange_config *best,
                                      float *bestMs)
{
    using namespace rfi;
    if (!ctx || trials < 1 || trials > 1000) {
        set_error("rf_tune_exchange: NULL context or trials outside 1..1000");
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    RF_CUDA(cudaStreamSynchronize(s));
    if (ctx->pending) {
        if (rf_status st = sync_state(ctx)) (void)st;
    }
    DevState saved;
    RF_CUDA(cudaMemcpy(&saved, ctx->dev, sizeof saved, cudaMemcpyDeviceToHost));
    if (saved.outCount == 0) {
        set_error("rf_tune_exchange: the out-queue is empty; emit a representative round first");
        return RF_ERR_ARG;
    }
    ScatterChoice v[kMaxVariants];
    const int nv = scatter_variants(ctx->itemBytes, v);
    // room for the smallest tile's histograms up front
    const uint32_t oldK = ctx->reqScatterK;
    const int oldS = ctx->reqScatterBlocks, oldC = ctx->reqCountBlocks;
    if (rf_status st = apply_config(ctx, v[nv - 1].k, 0, 0)) return st;

    cudaEvent_t e0, e1;
    RF_CUDA(cudaEventCreate(&e0));
    RF_CUDA(cudaEventCreate(&e1));
    float bestT = -1.0f;
    uint32_t bestK = v[0].k;
    int bestGrid = 0;
    rf_status st = RF_OK;
    for (int i = 0; i < nv && st == RF_OK; ++i) {
        const size_t smem = scatter_layout(256u * v[i].k, ctx->itemBytes, ctx->numRanks).total;
        int perSM = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perSM, v[i].fn, kBlock, smem) != cudaSuccess || perSM < 1)
            continue;
        const int grids[3] = {ctx->numSMs, 2 * ctx->numSMs, perSM * ctx->numSMs};
        for (int j = 0; j < 3 && st == RF_OK; ++j) {
            if (j == 1 && grids[1] >= grids[2]) continue;
            if (j == 2 && grids[2] == grids[0]) continue;
            st = apply_config(ctx, v[i].k, grids[j], 0);
            float tmin = -1.0f;
            for (uint32_t t = 0; t <= trials && st == RF_OK; ++t) {
                if (cudaMemsetAsync(ctx->count, 0, (size_t)ctx->numRanks * sizeof(uint32_t), s) != cudaSuccess ||
                    cudaEventRecord(e0, s) != cudaSuccess) {
                    st = cuda_fail(cudaGetLastError(), "rf_tune_exchange");
                    break;
                }
                st = launch_partition(ctx, s);
                if (st != RF_OK) break;
                if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                    st = cuda_fail(cudaGetLastError(), "rf_tune_exchange");
                    break;
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (t > 0 && (tmin < 0.0f || ms < tmin)) tmin = ms;  // the first run is a warm-up
            }
            if (st == RF_OK && tmin >= 0.0f && (bestT < 0.0f || tmin < bestT)) {
                bestT = tmin;
                bestK = v[i].k;
                bestGrid = grids[j];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the out-queue is untouched; the incoming queue is left empty
    saved.numActive = 0ull;
    cudaMemset(ctx->count, 0, (size_t)ctx->numRanks * sizeof(uint32_t));
    cudaMemset(ctx->inOffset, 0, (size_t)(ctx->numRanks + 1) * sizeof(uint32_t));
    cudaMemcpy(ctx->dev, &saved, sizeof saved, cudaMemcpyHostToDevice);
    *ctx->host = saved;
    ctx->pending = false;
    if (st != RF_OK || bestT < 0.0f) {
        (void)apply_config(ctx, oldK, oldS, oldC);
        if (st == RF_OK) {
            set_error("rf_tune_exchange: no scatter variant fits the device");
            st = RF_ERR_ARG;
        }
        return st;
    }
    if (rf_status as = apply_config(ctx, bestK, bestGrid, 0)) return as;
    RF_CUDA(cudaDeviceSynchronize());
    if (best) rf_get_exchange_config(ctx, best);
    if (bestMs) *bestMs = bestT;
    return RF_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free stable partition (rf_partition_static).
//
// The same count / scan / scatter kernels as rf_exchange, run on caller
// buffers, with their scratch (device state, per-destination totals, per-tile
// histograms) in one file-scope device array instead of context allocations.
// ---------------------------------------------------------------------------
#include <mutex>

namespace rfi {
namespace {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // 8 MiB, held by every device that loads the library
constexpr size_t kStaticCountOff = 256;                   // after the device state
constexpr size_t kStaticHistOff = kStaticCountOff + RF_MAX_RANKS * sizeof(uint32_t);
static_assert(sizeof(DevState) <= kStaticCountOff, "device state fits its slot");
static_assert(kStaticHistOff % 256 == 0, "histograms start aligned");

static __device__ __align__(256) unsigned char g_partition_scratch[kStaticScratchBytes];

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_base[kStaticMaxDevices] = {};

__global__ void __launch_bounds__(kBlock) static_init_kernel(DevState *s, uint32_t *count, int32_t R,
                                                             unsigned long long n)
{
    for (int e = threadIdx.x; e < R; e += kBlock) count[e] = 0u;
    if (threadIdx.x == 0) {
        s->outCount = n;
        s->bad = 0ull;
        s->holes = 0ull;
        s->numActive = 0ull;
        s->status = 0u;
    }
}

__global__ void static_finish_kernel(const DevState *s, unsigned long long *stats)
{
    if (threadIdx.x == 0 && stats) {
        stats[0] = s->numActive;
        stats[1] = s->holes;
        stats[2] = s->bad;
        stats[3] = s->status;
    }
}

// Once per device, with that device current: the device address of the
// scratch array, and the shared-memory limit of every scatter variant.
rf_status static_setup(int dev, unsigned char **base)
{
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_base[dev]) {
        void *p = nullptr;
        RF_CUDA(cudaGetSymbolAddress(&p, g_partition_scratch));
        int optin = 0;
        RF_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        for (uint32_t bytes : {16u, 32u, 48u, 64u, 128u, 80u, 160u, 512u}) {
            ScatterChoice v[kMaxVariants];
            const int m = scatter_variants(bytes, v);
            for (int i = 0; i < m; ++i)
                RF_CUDA(cudaFuncSetAttribute(v[i].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        }
        g_static_base[dev] = p;
    }
    *base = static_cast<unsigned char *>(g_static_base[dev]);
    return RF_OK;
}

}  // namespace
}  // namespace rfi

extern "C" rf_status rf_partition_static(const void *items, const int32_t *dest, uint64_t n, uint32_t itemBytes,
                                         int32_t numRanks, void *itemsOut, uint32_t *offsetsOut,
                                         unsigned long long *statsOut, void *stream)
{
    using namespace rfi;
    if (numRanks < 1 || numRanks > RF_MAX_RANKS || itemBytes == 0 || itemBytes % 16 ||
        itemBytes > RF_MAX_ITEM_BYTES || n > RF_MAX_CAPACITY || !offsetsOut || (n && (!items || !dest || !itemsOut))) {
        set_error("rf_partition_static: bad arguments (numRanks 1..%d, itemBytes a multiple of 16 up to %u, "
                  "n below 2^31, non-NULL buffers)", RF_MAX_RANKS, RF_MAX_ITEM_BYTES);
        return RF_ERR_ARG;
    }
    // The scatter stages input tiles with bulk copies and stores 16-byte
    // vectors: both item buffers must be 16-byte aligned, and they must not
    // overlap (other CTAs write output while a tile is still being read).
    const uintptr_t pi = reinterpret_cast<uintptr_t>(items), po = reinterpret_cast<uintptr_t>(itemsOut);
    const uint64_t span = n * (uint64_t)itemBytes;
    if (n && (((pi | po) & 15u) || (reinterpret_cast<uintptr_t>(dest) & 3u) ||
              (reinterpret_cast<uintptr_t>(statsOut) & 7u) || (pi < po + span && po < pi + span))) {
        set_error("rf_partition_static: items and itemsOut must be 16-byte aligned and must not overlap, dest "
                  "4-byte and statsOut 8-byte aligned");
        return RF_ERR_ARG;
    }
    if (reinterpret_cast<uintptr_t>(offsetsOut) & 3u) {
        set_error("rf_partition_static: offsetsOut must be 4-byte aligned");
        return RF_ERR_ARG;
    }
    const ScatterChoice c = pick_scatter(itemBytes);
    const uint32_t tileItems = 256u * c.k;
    const uint64_t tiles = (n + tileItems - 1) / tileItems;
    const uint64_t maxTiles = tiles < 4 ? 4 : (tiles + 3) / 4 * 4;
    const uint64_t histBytes = (uint64_t)numRanks * maxTiles * sizeof(uint32_t);
    if (kStaticHistOff + histBytes > kStaticScratchBytes) {
        set_error("rf_partition_static: %llu items over %d ranks need %llu bytes of scratch; the static "
                  "scratch holds %zu (numRanks x ceil(n / %u) x 4 bytes must stay below %zu)",
                  (unsigned long long)n, numRanks, (unsigned long long)(kStaticHistOff + histBytes),
                  kStaticScratchBytes, tileItems, kStaticScratchBytes - kStaticHistOff);
        return RF_ERR_ARG;
    }
    int dev = 0;
    RF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kStaticMaxDevices) {
        set_error("rf_partition_static: device %d beyond the %d supported", dev, kStaticMaxDevices);
        return RF_ERR_ARG;
    }
    unsigned char *base = nullptr;
    if (rf_status st = static_setup(dev, &base)) return st;

    const size_t smem = scatter_layout(tileItems, itemBytes, numRanks).total;
    int numSMs = 0, perSM = 0, cperSM = 0;
    RF_CUDA(cudaDeviceGetAttribute(&numSMs, cudaDevAttrMultiProcessorCount, dev));
    RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perSM, c.fn, kBlock, smem));
    RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cperSM, count_kernel, kBlock,
                                                          (size_t)numRanks * sizeof(uint32_t)));
    if (perSM < 1) {
        set_error("rf_partition_static: scatter tile does not fit on an SM (%zu bytes of shared memory)", smem);
        return RF_ERR_ARG;
    }
    ExArgs a;
    a.out = items;
    a.dest = dest;
    a.in = itemsOut;
    a.inOffset = offsetsOut;
    a.count = reinterpret_cast<uint32_t *>(base + kStaticCountOff);
    a.tileHist = reinterpret_cast<uint32_t *>(base + kStaticHistOff);
    a.state = reinterpret_cast<DevState *>(base);
    a.capacity = n;
    a.tileItems = tileItems;
    a.maxTiles = (uint32_t)maxTiles;
    a.itemBytes = itemBytes;
    a.numRanks = numRanks;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int mt = (int)maxTiles;
    const int cb = numSMs * (cperSM < 1 ? 1 : cperSM);
    const int sb = numSMs * perSM;
    static_init_kernel<<<1, kBlock, 0, s>>>(a.state, a.count, numRanks, n);
    RF_LAUNCHED("static_init_kernel");
    count_kernel<<<cb < mt ? cb : mt, kBlock, (size_t)numRanks * sizeof(uint32_t), s>>>(a);
    RF_LAUNCHED("count_kernel");
    scan_kernel<<<numRanks, kBlock, 0, s>>>(a);
    RF_LAUNCHED("scan_kernel");
    c.fn<<<sb < mt ? sb : mt, kBlock, smem, s>>>(a);
    RF_LAUNCHED("scatter_kernel");
    static_finish_kernel<<<1, 32, 0, s>>>(a.state, statsOut);
    RF_LAUNCHED("static_finish_kernel");
    return RF_OK;
}
