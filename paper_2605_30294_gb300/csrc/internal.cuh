// Internal declarations shared by the librafi_gb.so translation units:
// the context layout, error and launch bookkeeping, and thin inline-PTX
// wrappers (mbarrier, bulk async copy) used by the exchange kernels.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <functional>
#include <string>
#include <cstdint>
#include <cstdio>
#include <string>

#include "rafi.h"

namespace rfi {

// Device-resident state of one context.  The exchange's wrap-up kernel
// copies the per-exchange counters into the last* fields and clears the
// accumulators; the host reads the struct back after each exchange.
struct DevState {
    unsigned long long outCount;   // append counter of the out-queue
    unsigned long long bad;        // slots with an invalid destination (this exchange)
    unsigned long long holes;      // slots with destination -1 (this exchange)
    unsigned long long numActive;  // items delivered by the last exchange
    unsigned long long lastEmitted, lastDropped, lastBad, lastHoles;
    unsigned long long exchanges, totalDelivered, totalDropped;
    unsigned long long scratch;    // one-word scratch (append reservations)
    unsigned int status;           // RF_DEV_* bits, sticky until the host reads them
    unsigned int pad;
};

enum : unsigned int { RF_DEV_TIMEOUT = 1u };

// Upper bound on any spin-wait, in SM clock cycles (about half a second at
// 2 GHz); a wait that runs out sets RF_DEV_TIMEOUT and the kernel returns.
constexpr long long kSpinLimitCycles = 1000000000ll;

// Default largest round whose destination counts the persistent kernel's
// scatter pushes ahead (steps on arrival), in items.
constexpr uint32_t kPushMaxDefault = 1u << 16;

// Default rank skew of the persistent kernel's large-round ranges, in 1/256.
constexpr uint32_t kRankSkewDefault = 10u;

}  // namespace rfi

struct rf_ctx {
    int device = 0;
    int32_t numRanks = 0;
    uint32_t itemBytes = 0;
    uint64_t capacity = 0;
    uint32_t tileItems = 0;  // items per exchange tile
    uint32_t maxTiles = 0;   // tiles for a full queue, rounded up to a multiple of 4
    int numSMs = 0;
    int countBlocks = 0, scatterBlocks = 0;
    size_t scatterSmem = 0;

    void *in = nullptr;
    void *out = nullptr;
    int32_t *dest = nullptr;
    bool callerQueues = false;  // in, out and dest belong to the caller (rf_create_with_buffers)
    uint32_t *inOffset = nullptr;  // numRanks + 1
    uint32_t *count = nullptr;     // numRanks
    uint32_t *tileHist = nullptr;  // numRanks x maxTiles, digit-major
    uint32_t tileHistTiles = 0;    // tiles tileHist has room for
    uint32_t reqScatterK = 0;      // requested exchange configuration (0: default)
    int reqScatterBlocks = 0, reqCountBlocks = 0;
    rfi::DevState *dev = nullptr;
    rfi::DevState *host = nullptr;  // pinned mirror of *dev
    void *staging = nullptr;        // lazily allocated: capacity items (host-memory runs)
    unsigned long long *stagingCount = nullptr;
    cudaStream_t copyStream = nullptr;     // lazily created: copies in that overlap a run's kernel
    cudaStream_t copyOutStream = nullptr;  // and copies out
    cudaEvent_t copyDone[2] = {};
    unsigned long long *progressHost = nullptr;  // page-locked, mapped: a running launch's retired count
    unsigned long long *progressDev = nullptr;   // its device address

    cudaStream_t lastStream = nullptr;
    bool pending = false;  // an exchange's read-back has not been waited for

    void *roundsScratch = nullptr;  // lazily allocated scratch of the persistent round kernel
    void *loopState = nullptr;      // lazily allocated: rounds / forwarded / limit of the graph loop
    void *loopExec = nullptr;       // a kept graph loop (cudaGraphExec_t) and its graph, with its key
    void *loopGraph = nullptr;
    std::string loopKey;
    unsigned long long loopLaunchesPerRound = 0, loopLaunchesOnce = 0;
    size_t roundsScratchBytes = 0;

    uint32_t *zipfThr = nullptr;  // numRanks words: Zipf table of the microbenchmark
    double zipfS = -1.0;           // exponent the table was built for

    // per policy (RF_POLICY_*): the form a tuned run uses and the persistent kernel's shape
    int32_t batchedForm[3] = {RF_FORM_PERSISTENT, RF_FORM_PERSISTENT, RF_FORM_PERSISTENT};
    int32_t batchedShape[3] = {0, 0, 0};
    unsigned long long waitLimitCycles = 0;  // bound of the persistent kernel's barrier waits (0: kSpinLimitCycles)
    uint32_t missingArrivals = 0;            // > 0 only to exercise the timeout path
    uint32_t pushMax = rfi::kPushMaxDefault;  // rf_set_push_limit
    uint32_t rankSkew = rfi::kRankSkewDefault;  // rf_set_rank_skew

    bool timing = false;
    unsigned pendingSlots = 0;  // timing slots recorded since the last read-back
    cudaEvent_t ev[10] = {};
    rf_phase_times times = {};
};

namespace rfi {

extern std::atomic<unsigned long long> g_launches;

void set_error(const char *fmt, ...);
rf_status cuda_fail(cudaError_t e, const char *what);

inline void count_launch(unsigned long long k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

#define RF_CUDA(call)                                       \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return rfi::cuda_fail(e_, #call); \
    } while (0)

#define RF_LAUNCHED(name)                                       \
    do {                                                        \
        rfi::count_launch();                                    \
        cudaError_t e_ = cudaGetLastError();                    \
        if (e_ != cudaSuccess) return rfi::cuda_fail(e_, name); \
    } while (0)

// Makes the context's device current for the scope of an entry point.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Read back the device state of the last exchange (waits for its stream)
// and translate the counters into a status.
rf_status sync_state(rf_ctx *ctx);

// Launch count / scan / scatter / wrap-up for the context's out-queue.
rf_status launch_exchange(rf_ctx *ctx, cudaStream_t s);

// Tile size and grid shapes of the exchange from the context's request (or
// the defaults), and room for the per-tile histograms of that tile.
rf_status configure_exchange(rf_ctx *ctx);
rf_status ensure_tile_hist(rf_ctx *ctx);

// The graph form of the round loop: `round` enqueues one round's kernels
// (work, then the exchange) on the stream it is given; they are captured
// once into the body of a CUDA graph while node that repeats them, with no
// host round trip, while the exchange reports active items and fewer than
// maxRounds rounds have run.  Starts from the context's last exchange (which
// must be enqueued on s before); waits for s.  *rounds, *forwarded (host).
// prologue (may be empty) enqueues the kernels that seed the queue and its
// first exchange; they run in the graph before the loop.  With a key, the
// instantiated graph is kept in the context and relaunched while the key
// (every pointer and value the captured kernels take) is unchanged.
rf_status run_graph_loop(rf_ctx *ctx, cudaStream_t s, uint32_t maxRounds,
                         const std::function<rf_status(cudaStream_t)> &round, uint64_t *rounds, uint64_t *forwarded,
                         const std::function<rf_status(cudaStream_t)> &prologue = {}, const void *key = nullptr,
                         size_t keyBytes = 0);
// Release a kept graph loop (before the context's buffers change or go).
void drop_graph_loop(rf_ctx *ctx);

// The persistent kernel's shapes of each policy (defined beside the policy):
// write at most cap {block, itemsPerThread, ctasPerSM} triples, return the count.
int c1_shapes(int32_t *out, int32_t cap);
int c2_shapes(int32_t *out, int32_t cap);
int c4_shapes(int32_t *out, int32_t cap);

// Allocate ctx->staging (capacity items) on first use.
rf_status ensure_staging(rf_ctx *ctx);

// Create ctx->copyStream, ctx->copyOutStream, the two events and the mapped
// progress word once.
rf_status ensure_copy_stream(rf_ctx *ctx);

// Allocate (or grow) ctx->roundsScratch to at least `bytes` (zeroed).
rf_status ensure_rounds_scratch(rf_ctx *ctx, size_t bytes);

// Per-phase timing helpers (no-ops unless ctx->timing).
void time_begin(rf_ctx *ctx, int slot, cudaStream_t s);
void time_end(rf_ctx *ctx, int slot, cudaStream_t s);
void time_collect(rf_ctx *ctx);  // after a stream sync: accumulate recorded pairs

enum TimeSlot { kTimeCount = 0, kTimeScan = 1, kTimeScatter = 2, kTimeWork = 3, kTimeRounds = 4, kTimeSlots = 5 };

// ---------------------------------------------------------------------
// Inline PTX: mbarrier and bulk asynchronous copy global -> shared.
// ---------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global memory into this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dstSmem, const void *srcGlobal, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dstSmem)),
        "l"(srcGlobal), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar` to complete, for at most kSpinLimitCycles.
// Returns false (and the caller must record a timeout) if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kSpinLimitCycles) return false;
    }
    return true;
}

// Scalar bricks with a one-voxel halo (rf_c0_make_bricks) hold x-y quads:
// element (x, y, z) is the float4 {v(x, y), v(x+1, y), v(x, y+1), v(x+1, y+1)}
// of plane z, every index clamped to the volume, so the eight corners of a
// trilinear sample take two 16-byte loads.  jx, jy: brick-local indices of the
// lower x and y corner; z0, z1: the two planes; f: the fractions.  The blend
// runs in x, then y, then z.
__device__ __forceinline__ float quad_trilinear(const float4 *__restrict__ brick, int32_t S, int32_t jx, int32_t jy,
                                                int32_t z0, int32_t z1, const float f[3])
{
    const float4 q0 = __ldg(brick + ((size_t)z0 * S + jy) * S + jx);
    const float4 q1 = __ldg(brick + ((size_t)z1 * S + jy) * S + jx);
    const float gx = 1.0f - f[0], gy = 1.0f - f[1], gz = 1.0f - f[2];
    const float c00 = q0.x * gx + q0.y * f[0];
    const float c10 = q0.z * gx + q0.w * f[0];
    const float c01 = q1.x * gx + q1.y * f[0];
    const float c11 = q1.z * gx + q1.w * f[0];
    const float c0 = c00 * gy + c10 * f[1];
    const float c1 = c01 * gy + c11 * f[1];
    return c0 * gz + c1 * f[2];
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace rfi
