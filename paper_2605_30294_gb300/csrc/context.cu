// Host context (Sec. 3.4): creation, queue sizing (resizeRayQueues), the
// device interface (getDeviceInterface), host-side emits, read-back of the
// exchange state, checkpoint/resume, timing and error reporting.
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.cuh"

namespace rfi {

std::atomic<unsigned long long> g_launches{0};

namespace {
thread_local char g_err[512] = "";

__global__ void add_count_kernel(unsigned long long *counter, unsigned long long n)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *counter += n;
}

__global__ void set_state_kernel(DevState *s, unsigned long long numActive)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) s->numActive = numActive;
}
}  // namespace

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

rf_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return e == cudaErrorMemoryAllocation ? RF_ERR_OOM : RF_ERR_CUDA;
}


void time_begin(rf_ctx *ctx, int slot, cudaStream_t s)
{
    if (ctx->timing) cudaEventRecord(ctx->ev[2 * slot], s);
}

void time_end(rf_ctx *ctx, int slot, cudaStream_t s)
{
    if (!ctx->timing) return;
    cudaEventRecord(ctx->ev[2 * slot + 1], s);
    switch (slot) {
    case kTimeCount: ctx->times.countLaunches++; break;
    case kTimeScan: ctx->times.scanLaunches++; break;
    case kTimeScatter: ctx->times.scatterLaunches++; break;
    case kTimeWork: ctx->times.workLaunches++; break;
    case kTimeRounds: ctx->times.roundsLaunches++; break;
    default: break;
    }
    ctx->pendingSlots |= 1u << slot;
}

void time_collect(rf_ctx *ctx)
{
    if (!ctx->timing || !ctx->pendingSlots) return;
    for (int slot = 0; slot < kTimeSlots; ++slot) {
        if (!(ctx->pendingSlots & (1u << slot))) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev[2 * slot], ctx->ev[2 * slot + 1]) != cudaSuccess) continue;
        switch (slot) {
        case kTimeCount: ctx->times.countMs += ms; break;
        case kTimeScan: ctx->times.scanMs += ms; break;
        case kTimeScatter:
            ctx->times.scatterMs += ms;
            ctx->times.scatterItems += ctx->host->numActive;
            if (ctx->host->numActive >= (1ull << 20)) {
                ctx->times.scatterMsLarge += ms;
                ctx->times.scatterItemsLarge += ctx->host->numActive;
                ctx->times.scatterLaunchesLarge++;
            }
            break;
        case kTimeWork: ctx->times.workMs += ms; break;
        case kTimeRounds: ctx->times.roundsMs += ms; break;
        default: break;
        }
    }
    ctx->pendingSlots = 0;
}

rf_status sync_state(rf_ctx *ctx)
{
    if (ctx->pending) {
        RF_CUDA(cudaStreamSynchronize(ctx->lastStream));
        ctx->pending = false;
        time_collect(ctx);
    }
    const DevState *h = ctx->host;
    if (h->status & RF_DEV_TIMEOUT) {
        set_error("a bounded device-side wait gave up; the exchange is incomplete");
        return RF_ERR_TIMEOUT;
    }
    if (h->lastDropped) {
        set_error("%llu emits past capacity %llu were dropped", (unsigned long long)h->lastDropped,
                  (unsigned long long)ctx->capacity);
        return RF_ERR_OVERFLOW;
    }
    if (h->lastBad) {
        set_error("%llu items addressed to ranks outside [0, %d) were dropped", (unsigned long long)h->lastBad,
                  ctx->numRanks);
        return RF_ERR_BAD_DEST;
    }
    return RF_OK;
}

namespace {

void free_queues(rf_ctx *ctx)
{
    if (!ctx->callerQueues) {
        cudaFree(ctx->in);
        cudaFree(ctx->out);
        cudaFree(ctx->dest);
    }
    cudaFree(ctx->tileHist);
    cudaFree(ctx->staging);
    ctx->in = ctx->out = nullptr;
    ctx->dest = nullptr;
    ctx->tileHist = nullptr;
    ctx->tileHistTiles = 0;
    ctx->staging = nullptr;
}

rf_status alloc_queues(rf_ctx *ctx, uint64_t capacity)
{
    ctx->capacity = capacity;
    rf_status st = configure_exchange(ctx);
    if (st != RF_OK) return st;
    const size_t qbytes = (size_t)capacity * ctx->itemBytes;
    if (!ctx->callerQueues) {
        RF_CUDA(cudaMalloc(&ctx->in, qbytes));
        RF_CUDA(cudaMalloc(&ctx->out, qbytes));
        // padded to whole 16-byte units (+16 bytes) so a tile of destinations can be bulk-copied
        RF_CUDA(cudaMalloc(&ctx->dest, ((size_t)capacity + 3) / 4 * 16 + 16));
    }
    if (rf_status hs = ensure_tile_hist(ctx)) return hs;
    RF_CUDA(cudaMemset(ctx->inOffset, 0, (size_t)(ctx->numRanks + 1) * sizeof(uint32_t)));
    RF_CUDA(cudaMemset(ctx->count, 0, (size_t)ctx->numRanks * sizeof(uint32_t)));
    RF_CUDA(cudaMemset(ctx->dev, 0, sizeof(DevState)));
    memset(ctx->host, 0, sizeof(DevState));
    RF_CUDA(cudaDeviceSynchronize());
    return RF_OK;
}

rf_status check_ctx(rf_ctx *ctx, const char *fn)
{
    if (!ctx) {
        set_error("%s: NULL context", fn);
        return RF_ERR_ARG;
    }
    return RF_OK;
}

}  // namespace

rf_status ensure_rounds_scratch(rf_ctx *ctx, size_t bytes)
{
    if (ctx->roundsScratch && ctx->roundsScratchBytes >= bytes) return RF_OK;
    cudaFree(ctx->roundsScratch);
    ctx->roundsScratch = nullptr;
    ctx->roundsScratchBytes = 0;
    RF_CUDA(cudaMalloc(&ctx->roundsScratch, bytes));
    RF_CUDA(cudaMemset(ctx->roundsScratch, 0, bytes));
    ctx->roundsScratchBytes = bytes;
    return RF_OK;
}

rf_status ensure_staging(rf_ctx *ctx)
{
    if (ctx->staging) return RF_OK;
    RF_CUDA(cudaMalloc(&ctx->staging, (size_t)ctx->capacity * ctx->itemBytes));
    return RF_OK;
}

rf_status ensure_copy_stream(rf_ctx *ctx)
{
    if (!ctx->copyStream) RF_CUDA(cudaStreamCreateWithFlags(&ctx->copyStream, cudaStreamNonBlocking));
    if (!ctx->copyOutStream) RF_CUDA(cudaStreamCreateWithFlags(&ctx->copyOutStream, cudaStreamNonBlocking));
    for (cudaEvent_t &e : ctx->copyDone)
        if (!e) RF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (!ctx->progressHost) {
        RF_CUDA(cudaHostAlloc(reinterpret_cast<void **>(&ctx->progressHost), 64, cudaHostAllocMapped));
        RF_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void **>(&ctx->progressDev), ctx->progressHost, 0));
    }
    return RF_OK;
}

}  // namespace rfi

using namespace rfi;

extern "C" {

namespace {
rf_status create_ctx(int32_t numRanks, uint32_t itemBytes, uint64_t capacity, void *inBuf, void *outBuf,
                     int32_t *destBuf, rf_ctx **out);
}

rf_status rf_create(int32_t numRanks, uint32_t itemBytes, uint64_t capacity, rf_ctx **out)
{
    return create_ctx(numRanks, itemBytes, capacity, nullptr, nullptr, nullptr, out);
}

rf_status rf_create_with_buffers(int32_t numRanks, uint32_t itemBytes, uint64_t capacity, void *in, void *outQueue,
                                 int32_t *dest, rf_ctx **out)
{
    if (!in || !outQueue || !dest || ((uintptr_t)in & 15u) || ((uintptr_t)outQueue & 15u) ||
        ((uintptr_t)dest & 15u)) {
        set_error("rf_create_with_buffers: the queue buffers must be non-NULL and 16-byte aligned");
        if (out) *out = nullptr;
        return RF_ERR_ARG;
    }
    cudaPointerAttributes pa;
    for (const void *p : {static_cast<const void *>(in), static_cast<const void *>(outQueue),
                          static_cast<const void *>(dest)}) {
        if (cudaPointerGetAttributes(&pa, p) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
            (void)cudaGetLastError();
            set_error("rf_create_with_buffers: the queue buffers must be device memory");
            if (out) *out = nullptr;
            return RF_ERR_ARG;
        }
    }
    return create_ctx(numRanks, itemBytes, capacity, in, outQueue, dest, out);
}

namespace {
rf_status create_ctx(int32_t numRanks, uint32_t itemBytes, uint64_t capacity, void *inBuf, void *outBuf,
                     int32_t *destBuf, rf_ctx **out)
{
    if (!out) {
        set_error("rf_create: out is NULL");
        return RF_ERR_ARG;
    }
    *out = nullptr;
    if (numRanks < 1 || numRanks > RF_MAX_RANKS) {
        set_error("rf_create: numRanks %d outside [1, %d]", numRanks, RF_MAX_RANKS);
        return RF_ERR_ARG;
    }
    if (itemBytes == 0 || itemBytes % 16 || itemBytes > RF_MAX_ITEM_BYTES) {
        set_error("rf_create: itemBytes %u is not a multiple of 16 in [16, %u]", itemBytes, RF_MAX_ITEM_BYTES);
        return RF_ERR_ARG;
    }
    if (capacity == 0 || capacity > RF_MAX_CAPACITY) {
        set_error("rf_create: capacity %llu outside [1, 2^31 - 1]", (unsigned long long)capacity);
        return RF_ERR_ARG;
    }
    rf_ctx *ctx = new (std::nothrow) rf_ctx();
    if (!ctx) {
        set_error("rf_create: host allocation failed");
        return RF_ERR_OOM;
    }
    ctx->numRanks = numRanks;
    ctx->itemBytes = itemBytes;
    if (inBuf) {
        ctx->callerQueues = true;
        ctx->in = inBuf;
        ctx->out = outBuf;
        ctx->dest = destBuf;
    }
    rf_status st = RF_OK;
    do {
        cudaError_t e = cudaGetDevice(&ctx->device);
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaGetDevice"); break; }
        e = cudaDeviceGetAttribute(&ctx->numSMs, cudaDevAttrMultiProcessorCount, ctx->device);
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaDeviceGetAttribute"); break; }
        e = cudaMalloc(&ctx->inOffset, (size_t)(numRanks + 1) * sizeof(uint32_t));
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaMalloc(inOffset)"); break; }
        e = cudaMalloc(&ctx->count, (size_t)numRanks * sizeof(uint32_t));
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaMalloc(count)"); break; }
        e = cudaMalloc(&ctx->dev, sizeof(DevState));
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaMalloc(state)"); break; }
        e = cudaMalloc(&ctx->stagingCount, sizeof(unsigned long long));
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaMalloc(counter)"); break; }
        e = cudaMalloc(&ctx->zipfThr, (size_t)numRanks * sizeof(uint32_t));
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaMalloc(zipf)"); break; }
        e = cudaMallocHost(&ctx->host, sizeof(DevState));
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaMallocHost(state)"); break; }
        for (int i = 0; i < 2 * kTimeSlots && st == RF_OK; ++i) {
            e = cudaEventCreate(&ctx->ev[i]);
            if (e != cudaSuccess) st = cuda_fail(e, "cudaEventCreate");
        }
        if (st != RF_OK) break;
        st = alloc_queues(ctx, capacity);
    } while (0);
    if (st != RF_OK) {
        char keep[512];
        strncpy(keep, rf_last_error(), sizeof keep - 1);
        keep[sizeof keep - 1] = 0;
        rf_destroy(ctx);
        set_error("%s", keep);
        return st;
    }
    *out = ctx;
    return RF_OK;
}
}  // namespace

rf_status rf_destroy(rf_ctx *ctx)
{
    if (!ctx) return RF_OK;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    drop_graph_loop(ctx);
    free_queues(ctx);
    cudaFree(ctx->inOffset);
    cudaFree(ctx->count);
    cudaFree(ctx->dev);
    cudaFree(ctx->stagingCount);
    cudaFree(ctx->zipfThr);
    cudaFree(ctx->roundsScratch);
    cudaFree(ctx->loopState);
    if (ctx->host) cudaFreeHost(ctx->host);
    for (cudaEvent_t e : ctx->copyDone)
        if (e) cudaEventDestroy(e);
    if (ctx->copyStream) cudaStreamDestroy(ctx->copyStream);
    if (ctx->copyOutStream) cudaStreamDestroy(ctx->copyOutStream);
    if (ctx->progressHost) cudaFreeHost(ctx->progressHost);
    for (int i = 0; i < 2 * kTimeSlots; ++i)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    delete ctx;
    return RF_OK;
}

rf_status rf_resize(rf_ctx *ctx, uint64_t capacity)
{
    if (rf_status st = check_ctx(ctx, "rf_resize")) return st;
    if (capacity == 0 || capacity > RF_MAX_CAPACITY) {
        set_error("rf_resize: capacity %llu outside [1, 2^31 - 1]", (unsigned long long)capacity);
        return RF_ERR_ARG;
    }
    if (ctx->callerQueues) {
        set_error("rf_resize: the queues belong to the caller (rf_create_with_buffers); create a new context");
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    RF_CUDA(cudaDeviceSynchronize());
    ctx->pending = false;
    drop_graph_loop(ctx);
    free_queues(ctx);
    return alloc_queues(ctx, capacity);
}

rf_status rf_get_device_queues(rf_ctx *ctx, rf_device_queues *out)
{
    if (rf_status st = check_ctx(ctx, "rf_get_device_queues")) return st;
    if (!out) {
        set_error("rf_get_device_queues: out is NULL");
        return RF_ERR_ARG;
    }
    out->in = ctx->in;
    out->out = ctx->out;
    out->dest = ctx->dest;
    out->outCount = &ctx->dev->outCount;
    out->inOffset = ctx->inOffset;
    out->capacity = ctx->capacity;
    out->itemBytes = ctx->itemBytes;
    out->numRanks = ctx->numRanks;
    return RF_OK;
}

rf_status rf_num_active(rf_ctx *ctx, uint64_t *out)
{
    if (rf_status st = check_ctx(ctx, "rf_num_active")) return st;
    if (!out) {
        set_error("rf_num_active: out is NULL");
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    rf_status st = sync_state(ctx);
    *out = ctx->host->numActive;
    return st;
}

rf_status rf_segment(rf_ctx *ctx, int32_t rank, uint64_t *offset, uint64_t *count)
{
    if (rf_status st = check_ctx(ctx, "rf_segment")) return st;
    if (rank < 0 || rank >= ctx->numRanks || !offset || !count) {
        set_error("rf_segment: rank %d outside [0, %d) or NULL output", rank, ctx->numRanks);
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    rf_status st = sync_state(ctx);
    uint32_t v[2] = {0, 0};
    RF_CUDA(cudaMemcpy(v, ctx->inOffset + rank, sizeof v, cudaMemcpyDeviceToHost));
    *offset = v[0];
    *count = v[1] - v[0];
    return st;
}

rf_status rf_stats(rf_ctx *ctx, rf_round_stats *out)
{
    if (rf_status st = check_ctx(ctx, "rf_stats")) return st;
    if (!out) {
        set_error("rf_stats: out is NULL");
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    rf_status st = sync_state(ctx);
    const DevState *h = ctx->host;
    out->numActive = h->numActive;
    out->emitted = h->lastEmitted;
    out->dropped = h->lastDropped;
    out->badDest = h->lastBad;
    out->holes = h->lastHoles;
    out->exchanges = h->exchanges;
    out->totalDelivered = h->totalDelivered;
    out->totalDropped = h->totalDropped;
    return st;
}

rf_status rf_push(rf_ctx *ctx, const void *items, const int32_t *dest, uint64_t n, int32_t hostMemory, void *stream)
{
    if (rf_status st = check_ctx(ctx, "rf_push")) return st;
    if (n && (!items || !dest)) {
        set_error("rf_push: NULL items or dest");
        return RF_ERR_ARG;
    }
    if (n > RF_MAX_CAPACITY) {
        set_error("rf_push: n %llu too large", (unsigned long long)n);
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long oc = 0;
    RF_CUDA(cudaMemcpyAsync(&oc, &ctx->dev->outCount, sizeof oc, cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaStreamSynchronize(s));
    const uint64_t room = oc < ctx->capacity ? ctx->capacity - oc : 0;
    const uint64_t fit = n < room ? n : room;
    const cudaMemcpyKind kind = hostMemory ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (fit) {
        RF_CUDA(cudaMemcpyAsync(static_cast<unsigned char *>(ctx->out) + (size_t)oc * ctx->itemBytes, items,
                                (size_t)fit * ctx->itemBytes, kind, s));
        RF_CUDA(cudaMemcpyAsync(ctx->dest + oc, dest, (size_t)fit * sizeof(int32_t), kind, s));
    }
    add_count_kernel<<<1, 32, 0, s>>>(&ctx->dev->outCount, n);
    RF_LAUNCHED("add_count_kernel");
    return RF_OK;
}

rf_status rf_snapshot(rf_ctx *ctx, void *itemsOut, uint32_t *offsetsOut, void *stream)
{
    if (rf_status st = check_ctx(ctx, "rf_snapshot")) return st;
    if (!itemsOut || !offsetsOut) {
        set_error("rf_snapshot: NULL output");
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    rf_status st = sync_state(ctx);
    if (st == RF_ERR_CUDA || st == RF_ERR_TIMEOUT) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t n = ctx->host->numActive;
    if (n) RF_CUDA(cudaMemcpyAsync(itemsOut, ctx->in, (size_t)n * ctx->itemBytes, cudaMemcpyDeviceToDevice, s));
    RF_CUDA(cudaMemcpyAsync(offsetsOut, ctx->inOffset, (size_t)(ctx->numRanks + 1) * sizeof(uint32_t),
                            cudaMemcpyDeviceToDevice, s));
    return RF_OK;
}

rf_status rf_restore(rf_ctx *ctx, const void *items, const uint32_t *offsets, uint64_t n, void *stream)
{
    if (rf_status st = check_ctx(ctx, "rf_restore")) return st;
    if (!offsets || (n && !items) || n > ctx->capacity) {
        set_error("rf_restore: NULL input or n %llu above capacity", (unsigned long long)n);
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    rf_status st = sync_state(ctx);
    if (st == RF_ERR_CUDA) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n) RF_CUDA(cudaMemcpyAsync(ctx->in, items, (size_t)n * ctx->itemBytes, cudaMemcpyDeviceToDevice, s));
    RF_CUDA(cudaMemcpyAsync(ctx->inOffset, offsets, (size_t)(ctx->numRanks + 1) * sizeof(uint32_t),
                            cudaMemcpyDeviceToDevice, s));
    set_state_kernel<<<1, 32, 0, s>>>(ctx->dev, n);
    RF_LAUNCHED("set_state_kernel");
    ctx->host->numActive = n;
    return RF_OK;
}

rf_status rf_set_timing(rf_ctx *ctx, int32_t enable)
{
    if (rf_status st = check_ctx(ctx, "rf_set_timing")) return st;
    ctx->timing = enable != 0;
    ctx->pendingSlots = 0;
    return RF_OK;
}

rf_status rf_get_timing(rf_ctx *ctx, rf_phase_times *out, int32_t reset)
{
    if (rf_status st = check_ctx(ctx, "rf_get_timing")) return st;
    if (!out) {
        set_error("rf_get_timing: out is NULL");
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    rf_status st = sync_state(ctx);
    *out = ctx->times;
    if (reset) memset(&ctx->times, 0, sizeof ctx->times);
    return st;
}

rf_status rf_set_wait_limits(rf_ctx *ctx, uint64_t spinCycles, uint32_t missingArrivals)
{
    if (rf_status st = check_ctx(ctx, "rf_set_wait_limits")) return st;
    if (spinCycles > (1ull << 40) || missingArrivals > 1024u) {
        set_error("rf_set_wait_limits: spinCycles above 2^40 or missingArrivals above 1024");
        return RF_ERR_ARG;
    }
    ctx->waitLimitCycles = spinCycles;
    ctx->missingArrivals = missingArrivals;
    return RF_OK;
}

rf_status rf_set_push_limit(rf_ctx *ctx, uint64_t maxItems)
{
    if (rf_status st = check_ctx(ctx, "rf_set_push_limit")) return st;
    if (maxItems > 0xFFFFFFFFull) {
        set_error("rf_set_push_limit: %llu items above 2^32 - 1", (unsigned long long)maxItems);
        return RF_ERR_ARG;
    }
    ctx->pushMax = (uint32_t)maxItems;
    return RF_OK;
}

rf_status rf_get_push_limit(rf_ctx *ctx, uint64_t *maxItems)
{
    if (rf_status st = check_ctx(ctx, "rf_get_push_limit")) return st;
    if (!maxItems) {
        set_error("rf_get_push_limit: maxItems is NULL");
        return RF_ERR_ARG;
    }
    *maxItems = ctx->pushMax;
    return RF_OK;
}

rf_status rf_set_rank_skew(rf_ctx *ctx, uint32_t skew)
{
    if (rf_status st = check_ctx(ctx, "rf_set_rank_skew")) return st;
    if (skew > 32u) {
        set_error("rf_set_rank_skew: skew %u above 32", skew);
        return RF_ERR_ARG;
    }
    ctx->rankSkew = skew;
    return RF_OK;
}

rf_status rf_get_rank_skew(rf_ctx *ctx, uint32_t *skew)
{
    if (rf_status st = check_ctx(ctx, "rf_get_rank_skew")) return st;
    if (!skew) {
        set_error("rf_get_rank_skew: skew is NULL");
        return RF_ERR_ARG;
    }
    *skew = ctx->rankSkew;
    return RF_OK;
}

rf_status rf_rounds_shapes(int32_t policy, int32_t *count, int32_t *shapes, int32_t cap)
{
    if (!count || cap < 0 || (cap > 0 && !shapes)) {
        set_error("rf_rounds_shapes: NULL count or shapes");
        return RF_ERR_ARG;
    }
    int n = -1;
    if (policy == RF_POLICY_MICROBENCH) n = c1_shapes(shapes, cap);
    else if (policy == RF_POLICY_STREAMLINES) n = c2_shapes(shapes, cap);
    else if (policy == RF_POLICY_TRANSPORT) n = c4_shapes(shapes, cap);
    if (n < 0) {
        set_error("rf_rounds_shapes: unknown policy %d", policy);
        return RF_ERR_ARG;
    }
    *count = n;
    return RF_OK;
}

rf_status rf_set_batched_config(rf_ctx *ctx, int32_t policy, int32_t form, int32_t shape)
{
    if (rf_status st = check_ctx(ctx, "rf_set_batched_config")) return st;
    int32_t n = 0;
    if (rf_rounds_shapes(policy, &n, nullptr, 0) != RF_OK) return RF_ERR_ARG;
    if (form < RF_FORM_HOST_LOOP || form > RF_FORM_GRAPH || shape < 0 || shape >= n) {
        set_error("rf_set_batched_config: form %d or shape %d (of %d) out of range", form, shape, n);
        return RF_ERR_ARG;
    }
    ctx->batchedForm[policy] = form;
    ctx->batchedShape[policy] = shape;
    return RF_OK;
}

rf_status rf_get_batched_config(rf_ctx *ctx, int32_t policy, int32_t *form, int32_t *shape)
{
    if (rf_status st = check_ctx(ctx, "rf_get_batched_config")) return st;
    if (policy < RF_POLICY_MICROBENCH || policy > RF_POLICY_TRANSPORT) {
        set_error("rf_get_batched_config: unknown policy %d", policy);
        return RF_ERR_ARG;
    }
    if (form) *form = ctx->batchedForm[policy];
    if (shape) *shape = ctx->batchedShape[policy];
    return RF_OK;
}

uint64_t rf_launch_count(void) { return g_launches.load(); }

const char *rf_last_error(void) { return g_err; }

}  // extern "C"
