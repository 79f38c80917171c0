/*
 * rafi.h -- C ABI of librafi_gb.so: device-local work forwarding between
 * logical ranks on one GB300 (sm_103a).
 *
 * The paper's host context (Sec. 3.4) is created over a GPU and an MPI
 * communicator and offers three calls: resizeRayQueues(N),
 * getDeviceInterface() and forwardRays().  Here the communicator is replaced
 * by a count of logical ranks that all live in this GPU's memory: each rank
 * owns one contiguous segment of a shared incoming queue, and forwardRays()
 * (rf_exchange) is a device-side count / scan / stable scatter instead of a
 * sort plus MPI_Alltoall(v) (Sec. 4.2).
 *
 * Conventions for every entry point
 *   - Return an rf_status; nothing crosses the ABI as an exception.  On error
 *     rf_last_error() describes the most recent failure of the calling thread.
 *   - "device" pointers are CUDA global-memory pointers of the device that was
 *     current when the context was created; "host" pointers are ordinary
 *     (preferably pinned) host memory.  The caller keeps ownership of every
 *     pointer it passes; the context owns the queues it allocates.
 *   - stream is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  All work is stream-ordered on it; the collective barrier of
 *     forwardRays (Sec. 3.4) is plain stream order here.
 *   - Item sizes are multiples of 16 bytes (16-byte vector copies), at most
 *     RF_MAX_ITEM_BYTES.  Counts and offsets are below 2^31.
 */
#ifndef RAFI_H
#define RAFI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RF_MAX_ITEM_BYTES 512u
#define RF_MAX_RANKS 1024
#define RF_MAX_CAPACITY 0x7FFFFFFFull

typedef struct rf_ctx rf_ctx;

typedef enum rf_status {
    RF_OK = 0,
    RF_ERR_ARG = 1,        /* an argument is out of range or NULL where not allowed */
    RF_ERR_OOM = 2,        /* device or pinned host allocation failed */
    RF_ERR_CUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    RF_ERR_OVERFLOW = 4,   /* emits past capacity were dropped (Sec. 3.3); results valid */
    RF_ERR_BAD_DEST = 5,   /* items addressed to a rank outside [0, numRanks) were dropped */
    RF_ERR_MAX_ROUNDS = 6, /* a round loop hit its round limit with items still active */
    RF_ERR_TIMEOUT = 7,    /* a bounded device-side wait gave up; the kernel returned early */
    RF_ERR_STATE = 8       /* call not valid in the context's current state */
} rf_status;

/*
 * Device interface (Sec. 3.3, "DeviceInterface<T>"): a trivially copyable
 * struct that kernels receive by value.  Device-side helpers that read and
 * write it live in rafi_device.cuh (numIncoming, getIncoming, rankOf,
 * forward / emitOutgoing).
 *
 *   in        incoming items of all ranks, rank r's at [inOffset[r], inOffset[r+1])
 *   out       outgoing append queue (capacity items)
 *   dest      destination rank of each outgoing slot; -1 = empty slot (skipped)
 *   outCount  atomic append counter; it may run past capacity, and every emit
 *             at or past capacity is dropped (Sec. 3.3)
 *   inOffset  numRanks + 1 offsets; inOffset[numRanks] = items incoming in total
 */
typedef struct rf_device_queues {
    void *in;
    void *out;
    int32_t *dest;
    unsigned long long *outCount;
    const uint32_t *inOffset;
    uint64_t capacity;
    uint32_t itemBytes;
    int32_t numRanks;
} rf_device_queues;

/* What the most recent exchange saw, plus running totals since create. */
typedef struct rf_round_stats {
    uint64_t numActive;      /* items delivered (Sec. 4.2.3's reduce-add of received counts) */
    uint64_t emitted;        /* valid slots the out-queue held: min(outCount, capacity) */
    uint64_t dropped;        /* emits past capacity */
    uint64_t badDest;        /* slots whose destination was not -1 and outside [0, numRanks) */
    uint64_t holes;          /* slots with destination -1 */
    uint64_t exchanges;      /* exchanges since create */
    uint64_t totalDelivered; /* items delivered, summed over exchanges */
    uint64_t totalDropped;   /* dropped + badDest, summed over exchanges */
} rf_round_stats;

/* Accumulated device time per phase (CUDA events on the launching stream),
 * collected only while rf_set_timing(ctx, 1) is in effect. */
typedef struct rf_phase_times {
    double countMs, scanMs, scatterMs, workMs;
    uint64_t countLaunches, scanLaunches, scatterLaunches, workLaunches;
    uint64_t scatterItems;      /* items the timed scatter launches delivered */
    double scatterMsLarge;      /* the same, restricted to exchanges of >= 2^20 items */
    uint64_t scatterItemsLarge;
    uint64_t scatterLaunchesLarge;
    double roundsMs;            /* persistent round kernels (batched form) */
    uint64_t roundsLaunches;
} rf_phase_times;

/* --- host context (Sec. 3.4) ------------------------------------------- */

/* Create a context on the current CUDA device: numRanks logical ranks
 * (1..RF_MAX_RANKS), items of itemBytes bytes (multiple of 16, <=
 * RF_MAX_ITEM_BYTES), queues of capacity items in total over all ranks
 * (1..RF_MAX_CAPACITY; Sec. 3.4 resizeRayQueues).  Allocates the in/out
 * queues, destinations, counters and exchange scratch on the device.
 * *out is set on success and must be released with rf_destroy. */
rf_status rf_create(int32_t numRanks, uint32_t itemBytes, uint64_t capacity, rf_ctx **out);

/* rf_create over queues the caller owns (for example torch tensors): in and
 * outQueue hold capacity x itemBytes bytes each, dest ((capacity + 3) / 4 *
 * 4 + 4) int32 entries; all device memory, 16-byte aligned, alive until
 * rf_destroy, which leaves them alone.  The context allocates only its
 * offsets, counters and scratch.  rf_resize is refused (RF_ERR_ARG).
 * RF_ERR_ARG for NULL, misaligned or non-device buffers. */
rf_status rf_create_with_buffers(int32_t numRanks, uint32_t itemBytes, uint64_t capacity, void *in, void *outQueue,
                                 int32_t *dest, rf_ctx **out);

/* Release every allocation of the context (synchronises the device). NULL is a no-op. */
rf_status rf_destroy(rf_ctx *ctx);

/* resizeRayQueues(N) (Sec. 3.4): reallocate for a new total capacity.
 * Queue contents are discarded; the context is left empty. */
rf_status rf_resize(rf_ctx *ctx, uint64_t capacity);

/* getDeviceInterface() (Sec. 3.4): fill *out with the device pointers kernels use. */
rf_status rf_get_device_queues(rf_ctx *ctx, rf_device_queues *out);

/* forwardRays() (Sec. 3.4, Sec. 4.2): deliver every item in the out-queue to
 * its destination rank's incoming segment, stably (items keep their emission
 * order within a destination), reset the append counter, and compute the
 * number of items now active.  Kernels: count per destination, exclusive
 * scan, shared-memory-bucketed scatter, wrap-up.
 * numActiveOut != NULL: waits for the stream and returns the count, with
 *   RF_ERR_OVERFLOW / RF_ERR_BAD_DEST if items were dropped (the count is
 *   still valid).
 * numActiveOut == NULL: returns without waiting; errors surface on the next
 *   rf_num_active / rf_stats. */
rf_status rf_exchange(rf_ctx *ctx, void *stream, uint64_t *numActiveOut);

/* Launch shape of rf_exchange: items per scatter tile (256 x K; the tile
 * is staged in shared memory), and the grid sizes of the scatter and count
 * kernels.  In rf_set_exchange_config a zero field means the default (the
 * largest tile of at most 64 KiB, and as many CTAs as fit on the device). */
typedef struct rf_exchange_config {
    uint32_t tileItems;
    int32_t scatterBlocks;
    int32_t countBlocks;
} rf_exchange_config;

rf_status rf_get_exchange_config(rf_ctx *ctx, rf_exchange_config *out);
/* RF_ERR_ARG if no scatter variant has that tile for the context's item
 * size (tiles of 256 x K items, K from {16, 8, 4} for 16-byte items, {8, 4,
 * 2} for 32, {4, 2, 1} for 48 and 64, {2, 1} for 128) or a grid is negative. */
rf_status rf_set_exchange_config(rf_ctx *ctx, const rf_exchange_config *cfg);

/* Autotuner: times count + scan + scatter of the current out-queue (left
 * untouched; fill it with a representative round first) for every scatter
 * tile of the item size and scatter grids of 1x, 2x and the resident number
 * of CTAs per SM, trials timed runs each after one warm-up (CUDA events on
 * stream), and keeps the fastest.  *best, *bestMs (nullable): the chosen
 * configuration and its time.  The incoming queue is left empty.
 * RF_ERR_ARG if the out-queue is empty or trials is outside 1..1000. */
rf_status rf_tune_exchange(rf_ctx *ctx, void *stream, uint32_t trials, rf_exchange_config *best, float *bestMs);

/* Total of the most recent exchange (numIncoming over all ranks, Sec. 3.3);
 * waits for that exchange's stream. */
rf_status rf_num_active(rf_ctx *ctx, uint64_t *out);

/* numIncoming for one rank (Sec. 3.3), on the host: its segment [offset, offset + count). */
rf_status rf_segment(rf_ctx *ctx, int32_t rank, uint64_t *offset, uint64_t *count);

/* Statistics of the most recent exchange and running totals (waits for the stream). */
rf_status rf_stats(rf_ctx *ctx, rf_round_stats *out);

/* emitOutgoing from the host (Sec. 3.3): append n items with destinations to
 * the out-queue.  items (n x itemBytes) and dest (n int32) are host memory
 * when hostMemory != 0, device memory otherwise.  Items past capacity are
 * dropped and reported by the next exchange. */
rf_status rf_push(rf_ctx *ctx, const void *items, const int32_t *dest, uint64_t n, int32_t hostMemory,
                  void *stream);

/* Checkpoint: copy the incoming queue (rf_num_active items) and its numRanks+1
 * offsets out of the context.  Device pointers; itemsOut holds capacity items. */
rf_status rf_snapshot(rf_ctx *ctx, void *itemsOut, uint32_t *offsetsOut, void *stream);

/* Resume: replace the incoming queue with n items (device) whose segments are
 * given by numRanks+1 offsets (device, offsets[numRanks] == n). */
rf_status rf_restore(rf_ctx *ctx, const void *items, const uint32_t *offsets, uint64_t n, void *stream);

/* Per-phase CUDA-event timing on/off; read and clear the accumulated times. */
rf_status rf_set_timing(rf_ctx *ctx, int32_t enable);
rf_status rf_get_timing(rf_ctx *ctx, rf_phase_times *out, int32_t reset);

/* Bounds of the persistent round kernels' grid-barrier waits on this context
 * (the batched form, rf_c1_run_batched and the batched streamline and
 * transport runs).  Every such wait gives up after spinCycles SM clock cycles
 * (0 restores the default of 10^9, about half a second), raises an abort flag
 * that every other CTA sees at its next wait, and the call returns
 * RF_ERR_TIMEOUT with the context still usable: the next call reseeds it.
 * missingArrivals (normally 0) makes each grid barrier wait for that many CTAs
 * beyond the grid, which never arrive, so that every wait runs out: a way to
 * drive the timeout path on a real GPU without any fault.  The paper has no
 * counterpart (its only failure mode is the dropped emit of Sec. 3.3).
 * RF_ERR_ARG for spinCycles above 2^40 or missingArrivals above 1024. */
rf_status rf_set_wait_limits(rf_ctx *ctx, uint64_t spinCycles, uint32_t missingArrivals);

/* --- batched form: forms, shapes and the autotuner's settings ------------ */

/* Workloads that run the persistent round kernel (policies). */
#define RF_POLICY_MICROBENCH 0 /* rf_c1_run_batched */
#define RF_POLICY_STREAMLINES 1 /* rf_c2_run */
#define RF_POLICY_TRANSPORT 2 /* rf_c4_render */

/* Forms of a run: the per-round host loop, all rounds in one persistent
 * cooperative kernel, the round's kernels in a CUDA graph whose conditional
 * while node repeats them; RF_FORM_TUNED (rf_c2_run / rf_c4_render's batched
 * argument) takes the form and shape set for the policy on the context. */
#define RF_FORM_HOST_LOOP 0
#define RF_FORM_PERSISTENT 1
#define RF_FORM_GRAPH 2
#define RF_FORM_TUNED 3

/* The persistent kernel's compiled shapes for a policy: *count receives how
 * many there are; shapes (host, 3 x cap int32, may be NULL) receives
 * {threads per CTA, items per thread per tile, resident CTAs per SM} for the
 * first min(count, cap).  Every shape computes the same rounds, bit for bit;
 * only the time differs.  RF_ERR_ARG for an unknown policy. */
rf_status rf_rounds_shapes(int32_t policy, int32_t *count, int32_t *shapes, int32_t cap);

/* The form and shape a context uses for a policy: form for RF_FORM_TUNED runs
 * (RF_FORM_HOST_LOOP, _PERSISTENT or _GRAPH; the microbenchmark's batched call
 * is always persistent), shape for every persistent run of the policy.
 * Defaults: persistent, shape 0.  The autotuner (autotune.py in the package)
 * times the candidates on a sample of the caller's run and sets the fastest.
 * RF_ERR_ARG for an unknown policy, form or shape. */
rf_status rf_set_batched_config(rf_ctx *ctx, int32_t policy, int32_t form, int32_t shape);
rf_status rf_get_batched_config(rf_ctx *ctx, int32_t policy, int32_t *form, int32_t *shape);

/* Counts pushed ahead, for persistent runs that step on arrival (the
 * microbenchmark's rf_c1_run_batched): when the next round holds at most
 * maxItems items, each round's scatter also adds every item's next
 * destination into the count row of the CTA that owns the item's slot in
 * that round, so the round skips its count pass and its first grid barrier.
 * Segment offsets and queue order are those of Sec. 4.2 either way; only the
 * time differs.  0 turns it off; the default is 2^16 items.  The kernel caps
 * the limit at (2^32 - 1) / CTAs - 1.  RF_ERR_ARG above 2^32 - 1. */
rf_status rf_set_push_limit(rf_ctx *ctx, uint64_t maxItems);
rf_status rf_get_push_limit(rf_ctx *ctx, uint64_t *maxItems);

/* Rank skew, for persistent runs that step on arrival: CTAs that share an SM
 * are served unevenly by its memory pipeline (the earlier-launched first), so
 * equal ranges finish at different times and the SM idles on its last CTA.
 * With skew > 0, rounds of at least 2^19 items give each CTA a range in
 * proportion to 256 + skew x (k - 1 - 2 rho), rho its launch order among the k
 * CTAs on its SM (read from %smid once per launch, at the cost of one grid
 * barrier).  Queue order is that of Sec. 4.2.1 for any partition of the
 * queue into CTA ranges, so only the time differs.  0 (equal ranges) up to
 * 32, default 10; RF_ERR_ARG above 32. */
rf_status rf_set_rank_skew(rf_ctx *ctx, uint32_t skew);
rf_status rf_get_rank_skew(rf_ctx *ctx, uint32_t *skew);

/* Kernels this library launched in this process so far (all contexts). */
uint64_t rf_launch_count(void);

/* Message of the calling thread's most recent error ("" if none). */
const char *rf_last_error(void);

/* --- allocation-free partition ------------------------------------------ */

/* Stable partition of n items by destination into caller buffers, without
 * allocating anything.  The paper has no counterpart to this entry point.
 *
 * It exists for callers that must not call cudaMalloc once they are
 * running: latency-critical loops whose memory budget is fixed at start-up
 * (an allocation can synchronise and stall the whole device), and hosts
 * whose own caching allocator already owns almost all device memory (a fresh
 * allocation can fail while the host's pool still has room).
 *
 * Result: the same as rf_push + rf_exchange on a context: itemsOut (device,
 * room for n items) receives the items grouped by destination, keeping their
 * input order within a destination; offsetsOut (device, numRanks + 1 words)
 * receives the segment offsets.  dest == -1 marks an empty slot (skipped);
 * other destinations outside [0, numRanks) are dropped.  statsOut (device,
 * 4 words, may be NULL) receives {delivered, empty slots, dropped, status}.
 * items (n x itemBytes) and dest (n int32) are device memory.  items and
 * itemsOut must be 16-byte aligned and must not overlap (no in-place call);
 * dest and offsetsOut must be 4-byte aligned, statsOut 8-byte aligned.  A
 * call that breaks one of these rules returns RF_ERR_ARG before any launch.
 *
 * Scratch: one file-scope device array of 8 MiB, which every device that
 * loads the library holds until the process exits.  numRanks x ceil(n /
 * tile) x 4 bytes (tile = 256 items for 256-byte items, up to 4096 items for
 * 16-byte items) must fit in 8 MiB - 4352 bytes; larger requests fail with
 * RF_ERR_ARG and say so.  The scratch is cleared at the start of each call.
 * Every call shares it: calls whose work may overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * The first call on a device looks up the array's device address and sets
 * kernel attributes (no allocation); make that first call before any stream
 * capture.  Asynchronous on stream; never calls cudaMalloc or cudaFree. */
rf_status rf_partition_static(const void *items, const int32_t *dest, uint64_t n, uint32_t itemBytes,
                              int32_t numRanks, void *itemsOut, uint32_t *offsetsOut,
                              unsigned long long *statsOut, void *stream);

/* --- forwarding microbenchmark (64-byte items) --------------------------- */

/* Destination laws of the microbenchmark work kernel. */
#define RF_C1_UNIFORM 0
#define RF_C1_ZIPF 1
#define RF_C1_NBR6 2

/* Zipf table for numRanks ranks and exponent s, on the host: thr[k] =
 * floor(2^32 * P(rank <= k)), rank k weighted (k+1)^-s, k = 0 .. numRanks-2;
 * sums in double, in increasing k. */
rf_status rf_c1_zipf_thresholds(int32_t numRanks, double s, uint32_t *thrHost);

/* Seed (the raygen step of Sec. 5.1): emit item i of items (device, n x 64
 * bytes) to rank i mod numRanks.  Follow with rf_exchange. */
rf_status rf_c1_seed(rf_ctx *ctx, const void *items, uint64_t n, void *stream);

/* One round of the per-rank work kernel over the incoming queue (64-byte
 * items, words w0..w15).  Each item draws r = Philox4x32-10(key {seed, 1},
 * counter {w0, w1, w15, hop}) (Salmon et al., SC'11).  r0 < ceil(0.1 * 2^32):
 * the item retires unchanged into retired (device, retiredCapacity items) at
 * index atomicAdd(retiredCount, 1) (device counter).  Otherwise r1 picks a
 * destination d by mode: RF_C1_UNIFORM floor(r1 * numRanks / 2^32);
 * RF_C1_ZIPF the first k with r1 < thr[k] of rf_c1_zipf_thresholds(numRanks,
 * zipfS), else numRanks - 1; RF_C1_NBR6 direction floor(r1 * 6 / 2^32) =
 * +x,-x,+y,-y,+z,-z from the item's rank on the torus gx x gy x gz (rank = x +
 * gx*(y + gy*z), wrapping).  The item becomes w14 = d, w13 ^= r2, w15 += 1 and
 * is forwarded to d.
 * deterministic != 0: out slot i holds incoming item i (destination -1 when it
 * retired), so queue order does not depend on scheduling; the out-queue must
 * be empty before the call. */
rf_status rf_c1_work(rf_ctx *ctx, uint32_t seed, uint32_t hop, int32_t mode, double zipfS, int32_t gx,
                     int32_t gy, int32_t gz, void *retired, unsigned long long *retiredCount,
                     uint64_t retiredCapacity, int32_t deterministic, void *stream);

/* The whole microbenchmark: seed, exchange, then { work (hop = round); exchange }
 * until no item is active (RF_ERR_MAX_ROUNDS after maxRounds rounds).
 * hostMemory == 0: items and retired are device buffers of n x 64 bytes.
 * hostMemory != 0: they are host buffers (pinned for speed); the items are
 *   copied into the empty out-queue and the retired items back, inside the call.
 * *retiredCountOut (host) = items retired; *rounds = work rounds run;
 * *forwarded = items delivered by the exchanges after work rounds (the seed
 * exchange excluded).  Waits for the stream before returning. */
rf_status rf_c1_run(rf_ctx *ctx, const void *items, uint64_t n, uint32_t seed, int32_t mode, double zipfS,
                    int32_t gx, int32_t gy, int32_t gz, void *retired, uint64_t *retiredCountOut,
                    int32_t deterministic, int32_t hostMemory, uint32_t maxRounds, void *stream,
                    uint64_t *rounds, uint64_t *forwarded);

/* rf_c1_run (device buffers) with the rounds in a CUDA graph: the seed and
 * its exchange, then a conditional while node repeating { work kernel;
 * exchange } on the device while items are active (the hop of each round
 * read from the device), with no host round trip per round.  Results and
 * errors as rf_c1_run. */
rf_status rf_c1_run_graph(rf_ctx *ctx, const void *items, uint64_t n, uint32_t seed, int32_t mode, double zipfS,
                          int32_t gx, int32_t gy, int32_t gz, void *retired, uint64_t *retiredCountOut,
                          int32_t deterministic, uint32_t maxRounds, void *stream, uint64_t *rounds,
                          uint64_t *forwarded);

/* Batched form of rf_c1_run: the seed as in rf_c1_run, then every work
 * round and exchange inside one persistent cooperative kernel, so no round
 * needs the host.  Per round: destination counts per CTA range, bounded grid
 * barrier, destination offsets and the next active count, stable scatter
 * (retirement is one more destination: the retired items land, stably, in
 * `retired`), bounded grid barrier.
 * stepOnArrival != 0: the scatter applies the next round's work step to each
 * item as it lands in its destination's segment, so an item crosses HBM once
 * per round; the seed exchange is the kernel's first scatter (it applies
 * round 0's step).  A run that stops at maxRounds scatters its last round
 * plainly, leaving the unstepped queue.
 * stepOnArrival == 0: the seed exchange runs first; each round's work step
 * reads and writes back every item in its queue slot before the scatter.
 * Queue order is deterministic either way: round k's incoming queue is the
 * one of rf_c1_run with deterministic != 0.  With hostMemory != 0 and a
 * page-locked (device-mapped) retired buffer the kernel writes the retired
 * items straight into it during the run; other host buffers are filled from
 * a device staging buffer after it.  The kernel runs in the shape set for
 * RF_POLICY_MICROBENCH on the context (rf_set_batched_config; shape 0 by
 * default: tiles of 512 items, 3 CTAs per SM).  Rounds of at most one tile
 * run on one CTA (the others return); with steps on arrival such rounds keep
 * the whole queue in that CTA's shared memory.  roundLog (device, 7 x roundLogCap
 * words, nullable) receives per round, as seen by CTA 0, the %globaltimer ns
 * at round start, end of its work step (or count), after the first barrier,
 * end of its scatter and after the second barrier, then the incoming and the
 * delivered item counts.  RF_ERR_TIMEOUT if a bounded wait gave up.
 * Other arguments and results as rf_c1_run. */
rf_status rf_c1_run_batched(rf_ctx *ctx, const void *items, uint64_t n, uint32_t seed, int32_t mode, double zipfS,
                            int32_t gx, int32_t gy, int32_t gz, void *retired, uint64_t *retiredCountOut,
                            int32_t hostMemory, int32_t stepOnArrival, uint32_t maxRounds, void *stream,
                            uint64_t *rounds, uint64_t *forwarded, unsigned long long *roundLog,
                            uint32_t roundLogCap);

/* Several independent runs of the microbenchmark (1 to 4) in one persistent
 * launch, steps on arrival: the batched form over several seed sets.  Run k
 * holds items [k n, (k + 1) n) of items (numRuns x n x 64 bytes, device or,
 * with hostMemory != 0, host memory); its item i starts at rank i mod
 * numRanks, as in a run of its own, and hops under modes[k] (host array of
 * numRuns laws; gx, gy, gz as rf_c1_run when a run is RF_C1_NBR6).  The runs
 * share the ranks' queues: a round's queue of rank r holds every run's items
 * bound for r, and the stable partition of Sec. 4.2.1, restricted to one run,
 * is that run's own partition, so each run's round queues and retirement
 * order are exactly those of rf_c1_run_batched on it alone.  Each run has a
 * retirement destination of its own: run k's retired items land, stably, in
 * retired slots [k n, (k + 1) n) (numRuns x n x 64 bytes; page-locked host
 * memory receives them during the run, other host memory after it).  With
 * hostMemory != 0 and a page-locked retired buffer the runs are launched one
 * after another instead (each as rf_c1_run_batched, reading its items in
 * place from a queue slot beyond the first n and retiring into a device
 * staging buffer): while run k executes, run k + 1's items are copied in and
 * run k's retired items copied out, as their slots become final, on two
 * streams of the context's own, so both directions of the host link work at
 * once; the results are the same, roundLog is not written.
 * Results (host): retiredCountsOut[k] and roundsOut[k] (nullable) per run,
 * *forwarded (nullable) the deliveries of all runs' work rounds.  The
 * context's capacity must hold numRuns x n items (below 2^31).  A launch that
 * stops at maxRounds (RF_ERR_MAX_ROUNDS) leaves a queue that no later call
 * resumes.  roundLog as rf_c1_run_batched, over the joint rounds.  RF_ERR_ARG
 * for 0 or more than 4 runs, a bad mode, a NULL array or a size above the
 * capacity; RF_ERR_TIMEOUT if a bounded wait gave up. */
rf_status rf_c1_run_batched_runs(rf_ctx *ctx, const void *items, uint64_t n, int32_t numRuns, uint32_t seed,
                                 const int32_t *modes, double zipfS, int32_t gx, int32_t gy, int32_t gz,
                                 void *retired, uint64_t *retiredCountsOut, int32_t hostMemory, uint32_t maxRounds,
                                 void *stream, uint64_t *roundsOut, uint64_t *forwarded,
                                 unsigned long long *roundLog, uint32_t roundLogCap);

/* --- absorption marching through bricks (48-byte rays) ------------------- */

/* Cut an N^3 float volume (device, x fastest) into (N/B)^3 bricks of
 * (B+2)^3 elements with a one-voxel halo.  Element (lx, ly, lz) is the x-y
 * quad {v(x, y), v(x+1, y), v(x, y+1), v(x+1, y+1)} of plane z, where (x, y,
 * z) = the brick's halo origin + (lx, ly, lz) and every index is clamped to
 * the volume (so the eight corners of a trilinear sample take two 16-byte
 * loads).  Brick of rank r = bx + nb*(by + nb*bz) at bricks + r*(B+2)^3*4
 * floats; bricks (device, (N/B)^3*(B+2)^3*4 floats) must be 16-byte aligned,
 * else RF_ERR_ARG, here and in the calls that read them. */
rf_status rf_c0_make_bricks(const float *volume, int32_t N, int32_t B, float *bricks, void *stream);

/* Raygen (Sec. 5.1 step 2): one primary ray per pixel of a W x H pinhole
 * camera cam (host, 12 floats: eye, corner, du, dv); a ray with a sample in
 * [0,N]^3 is forwarded to the brick holding its first sample, any other ray
 * writes T = 1 to image (device, W*H floats).  Follow with rf_exchange. */
rf_status rf_c0_raygen(rf_ctx *ctx, const float *cam, int32_t N, int32_t B, int32_t W, int32_t H,
                       float *image, void *stream);

/* Trace (Sec. 5.1 step 3, absorption only): every rank marches its incoming
 * rays through its brick at step 0.5 (tau += sigma * 0.5), forwarding a ray
 * to the next brick when a sample leaves its own, and writing T = expf(-tau)
 * to image[pixel] when the ray leaves the volume.  hopLog (device, W*H x
 * maxHops, nullable) records the ranks each pixel's ray visited, hopCount
 * (device, W*H) how many. */
rf_status rf_c0_march(rf_ctx *ctx, const float *bricks, int32_t N, int32_t B, float *image,
                      int32_t *hopLog, int32_t maxHops, int32_t *hopCount, void *stream);

/* The whole render: raygen, exchange, then { march; exchange } until no ray
 * is active (at most maxRounds rounds).  *rounds = march rounds run. */
rf_status rf_c0_render(rf_ctx *ctx, const float *bricks, const float *cam, int32_t N, int32_t B,
                       int32_t W, int32_t H, float *image, int32_t *hopLog, int32_t maxHops,
                       int32_t *hopCount, uint32_t maxRounds, void *stream, uint64_t *rounds);

/* rf_c0_render as a CUDA graph: raygen and its exchange, then a conditional
 * while node repeating { march; exchange } on the device while rays are
 * active, with no host round trip per round.  The instantiated graph stays
 * in the context and is relaunched while every argument is unchanged (a
 * changed argument, rf_resize or an exchange configuration rebuilds it).
 * Same arguments, results and errors as rf_c0_render. */
rf_status rf_c0_render_graph(rf_ctx *ctx, const float *bricks, const float *cam, int32_t N, int32_t B, int32_t W,
                             int32_t H, float *image, int32_t *hopLog, int32_t maxHops, int32_t *hopCount,
                             uint32_t maxRounds, void *stream, uint64_t *rounds);

/* Marching with each rank's brick staged whole in shared memory by one 3-D
 * tensor copy (TMA, cp.async.bulk.tensor), the alternative to the quad bricks
 * read through L1 (VoPaT's per-rank trace, Sec. 5.1).  Bricks come from
 * rf_c0_make_scalar_bricks: per rank (B+2)^3 scalars with a one-voxel halo,
 * each index clamped to the volume, rows padded to rf_c0_scalar_row(B) =
 * (B + 2) rounded up to a multiple of 4 floats (TMA copies rows of whole
 * 16-byte units); device memory, 16-byte aligned, R x row x (B+2)^2 floats.
 * A CTA takes up to 256 rays of one rank's incoming segment and marches them
 * from the staged brick with the same corners and float operations as
 * rf_c0_march, so the image is bit-identical.  The staged brick must fit in
 * one CTA's shared memory (B = 32: 166 KB); larger bricks get RF_ERR_ARG.
 * RF_ERR_CUDA if the driver offers no tensor-map encoder.  rf_c0_render_tma
 * is rf_c0_render with this march (no hop log), as the host loop (form
 * RF_FORM_HOST_LOOP) or with its rounds in a kept CUDA graph whose
 * conditional while node repeats them (RF_FORM_GRAPH, as rf_c0_render_graph). */
rf_status rf_c0_make_scalar_bricks(const float *volume, int32_t N, int32_t B, float *bricks, void *stream);
rf_status rf_c0_march_tma(rf_ctx *ctx, const float *scalarBricks, int32_t N, int32_t B, float *image, void *stream);
rf_status rf_c0_render_tma(rf_ctx *ctx, const float *scalarBricks, const float *cam, int32_t N, int32_t B, int32_t W,
                           int32_t H, float *image, int32_t form, uint32_t maxRounds, void *stream, uint64_t *rounds);

/* --- streamlines through bricks (32-byte particles) ------------------------ */

/* Particle: {x, y, z (float bits), id} {steps, hops, set, status}; status 1 =
 * left the grid, 2 = a step did not move it, 3 = maxSteps reached. */
#define RF_C2_EXITED 1
#define RF_C2_STALLED 2
#define RF_C2_MAXSTEPS 3

/* Cut an N^3 x 3 float vector field (device, index ((z*N + y)*N + x)*3 + c)
 * into (N/B)^3 bricks of (B+4)^3 elements with a two-voxel halo.  Element
 * (lx, ly, lz) holds 8 floats {vx, vy, vz, 0} of the voxel at the brick's
 * halo origin + (lx, ly, lz) and the same for the voxel one step further
 * along x, both clamped to the grid (so one 32-byte load gives both x corners
 * of a trilinear sample).  Brick of rank r = bx + nb*(by + nb*bz) at
 * bricks + r*(B+4)^3*8 floats; bricks (device, (N/B)^3*(B+4)^3*8 floats) must
 * be 32-byte aligned, else RF_ERR_ARG, here and in the calls that read them. */
rf_status rf_c2_make_bricks(const float *field, int32_t N, int32_t B, float *bricks, void *stream);

/* Seed (Sec. 5.4 "particles are released at predefined seed points"):
 * particle i at seeds[i] (device, n x 3 floats, inside [0,N)^3), id i, set
 * setIds[i] (device, nullable: 0), emitted to the rank owning its position.
 * The out-queue must be empty.  Follow with rf_exchange. */
rf_status rf_c2_seed(rf_ctx *ctx, const float *seeds, const uint32_t *setIds, uint64_t n, int32_t N, int32_t B,
                     void *stream);

/* One round of the per-rank trace kernel (Sec. 5.4): each incoming particle
 * takes RK4 steps of size h on the trilinear field of its rank's brick
 * (k1 = v(p), k2 = v(p + h/2 k1), k3 = v(p + h/2 k2), k4 = v(p + h k3),
 * p' = p + h/6 (k1 + 2 k2 + 2 k3 + k4)); it stops when it has made maxSteps
 * steps, a step does not move it, or it leaves [0,N)^3, and the stopped
 * particle is written to out[id] (device, outCapacity x 32 bytes).  It is
 * forwarded when a step enters another rank's brick (hops + 1), or to its own
 * rank after stepsPerRound steps (0: no such limit).  Out slot i holds
 * incoming particle i (destination -1 once stopped). */
rf_status rf_c2_trace(rf_ctx *ctx, const float *bricks, int32_t N, int32_t B, float h, uint32_t maxSteps,
                      uint32_t stepsPerRound, void *out, uint64_t outCapacity, void *stream);

/* Seed, exchange, then rounds of trace + exchange until no particle is
 * active.  batched == 0: the plain host loop (rf_c2_trace + rf_exchange per
 * round); batched == 1: all rounds in one persistent cooperative kernel (the
 * batched form of rf_c1_run_batched); batched == 2: the trace kernel and the
 * exchange kernels captured once into a CUDA graph whose conditional while
 * node repeats them on the device while particles are active; batched == 3
 * (RF_FORM_TUNED): the form set for RF_POLICY_STREAMLINES on the context
 * (rf_set_batched_config).  Persistent runs use the context's shape for the
 * policy.  out (device) receives every particle by id; *rounds = trace
 * rounds, *forwarded = particles delivered by them. */
rf_status rf_c2_run(rf_ctx *ctx, const float *bricks, const float *seeds, const uint32_t *setIds, uint64_t n,
                    int32_t N, int32_t B, float h, uint32_t maxSteps, uint32_t stepsPerRound, void *out,
                    int32_t batched, uint32_t maxRounds, void *stream, uint64_t *rounds, uint64_t *forwarded);

/* --- differentiable emission-absorption rendering (64-byte rays) ---------- */

/* Forward render through bricks made by rf_c0_make_bricks (halo 1): spp
 * jittered rays per pixel of a W x H camera cam (host, 12 floats), sample s
 * of pixel p aiming at (x + u, y + v) with u, v the top 24 bits of words 0
 * and 1 of Philox4x32-10(key {seed, 5}, counter {p, s, 0, 0}) / 2^24.
 * Samples at t0 + (k + 0.5) * 0.5; per sample e = expf(-sigma/2), alpha =
 * 1 - e, c = 20 sigma, C += (T alpha) c, T *= e (the Lander renderer's
 * emission-absorption model, Sec. 5.2, each ray carrying C and T across
 * bricks).  rayC (device, W*H*spp) receives every sample's C (the plain float
 * sum), image (device, W*H) the mean over a pixel's samples.  rayCLo (device,
 * W*H*spp, or NULL) receives the rounding error of each C, kept with Knuth's
 * error-free TwoSum, so that C + Clo is the exact sum of the float terms to
 * about 2^-48 relative; rf_c3_adjoint uses it to take exact suffixes. */
rf_status rf_c3_render(rf_ctx *ctx, const float *bricks, const float *cam, int32_t N, int32_t B, int32_t W, int32_t H,
                       int32_t spp, uint32_t seed, float *rayC, float *rayCLo, float *image, uint32_t maxRounds,
                       void *stream, uint64_t *rounds);

/* Adjoint of rf_c3_render: given rayC (and rayCLo, or NULL) from the forward
 * call and gradImage = dL/dimage (device, W*H), adds dL/dsigma to gradVolume
 * (device, N^3, x fastest; the caller zeroes it).  Adjoint rays carry their
 * forward C and dL/dC (= gradImage / spp) through the same bricks, recompute
 * T per brick and scatter dC/dsigma_k = T_k (0.5 e_k c_k + 20 alpha_k) - 0.5
 * S_{>k} with the trilinear weights, where the suffix S_{>k} = C - sum_{j<=k}
 * T_j alpha_j c_j is kept as a TwoSum pair starting from (C, Clo): exact up to
 * the rounding of the terms when rayCLo is given, else off by the rounding of
 * C itself.  Atomic adds: the summation order, not the value, depends on
 * scheduling. */
rf_status rf_c3_adjoint(rf_ctx *ctx, const float *bricks, const float *cam, int32_t N, int32_t B, int32_t W,
                        int32_t H, int32_t spp, uint32_t seed, const float *rayC, const float *rayCLo,
                        const float *gradImage, float *gradVolume, uint32_t maxRounds, void *stream,
                        uint64_t *rounds);

/* --- stochastic transport by delta tracking (64-byte paths) -------------- */

/* Render numViews views (cams: host, 12 floats each; sizes: host, {W, H}
 * each) at spp paths per pixel through bricks made by rf_c0_make_bricks
 * (halo 1) of an N^3 extinction grid with majorant sigmaMax (>= every
 * voxel).  Path s of global pixel gpix (pixels numbered view after view,
 * row-major) starts where its jittered ray (Philox key {seed, 9}) enters
 * the grid; event (bounce b, index e) draws r = Philox4x32-10(key {seed, 7},
 * counter {gpix, s, b, e}): free flight -logf(1 - u(r0)) / sigmaMax; leaving
 * the grid scores 1; a real collision (u(r1) sigmaMax < sigma) scatters when
 * u(r2) < 0.8 (Henyey-Greenstein g = 0.3 from u(r3) and word 0 of Philox
 * key {seed, 8}; more than 64 bounces score 0), else absorbs (score 0); a
 * null collision moves on with e + 1.  u(r) = top 24 bits / 2^24.  Paths are
 * forwarded to the rank owning their next tentative collision point (VoPaT,
 * Sec. 5.1, Fig. 1).  score (device, total pixels; the caller zeroes it)
 * receives the number of escaped paths per pixel.  batched: 0 host loop, 1
 * persistent kernel, 2 CUDA graph loop, 3 the form set for
 * RF_POLICY_TRANSPORT on the context, as rf_c2_run.  *rounds, *forwarded as
 * rf_c2_run. */
rf_status rf_c4_render(rf_ctx *ctx, const float *bricks, int32_t N, int32_t B, float sigmaMax, int32_t numViews,
                       const float *cams, const int32_t *sizes, int32_t spp, uint32_t seed, float *score,
                       int32_t batched, uint32_t maxRounds, void *stream, uint64_t *rounds, uint64_t *forwarded);

/* --- multi-phase exchange with three item types (Sec. 5.5) -------------- */

/* The communication pattern of the paper's distributed N-body code: three
 * contexts of different item types on one stream.  A particle context moves
 * 32-byte particles {x, y, z (uint32 fixed point on the periodic unit cube),
 * vx, vy, vz (int32), m, id}; a node context moves 64-byte nodes {M, X, Y, Z
 * (uint64: mass and mass-weighted coordinate sums), count, src, code (0 =
 * root, 1 + o = octant o), level, 4 pad words}; a request context moves
 * 16-byte requests {requester, target, code, level}.  All three have
 * numRanks = gx * gy * gz ranks (powers of two); rank of a position = the
 * top log2(g) bits of each coordinate, x fastest.  nodes (device) holds
 * numRanks x 9 x 5 uint64: per rank its root, then octants 0..7 (the bit
 * after the rank bits, x lowest), as {M, X, Y, Z, count}.
 * Every call is asynchronous on stream except rf_mp_step.  Errors: RF_ERR_ARG
 * for a context of the wrong item size, mismatched rank counts or devices, a
 * grid that is not gx x gy x gz powers of two or NULL buffers. */

/* Emit n particles (device, n x 32 bytes) into the particle context's
 * out-queue, each to the rank owning its position. */
rf_status rf_mp_seed(rf_ctx *particles, const void *items, uint64_t n, int32_t gx, int32_t gy, int32_t gz,
                     void *stream);
/* Migration: every incoming particle moves by its velocity (wrapping) and is
 * forwarded to the rank owning its new position. */
rf_status rf_mp_migrate(rf_ctx *particles, int32_t gx, int32_t gy, int32_t gz, void *stream);
/* Local trees of the incoming particles of every rank into nodes (exact). */
rf_status rf_mp_tree(rf_ctx *particles, int32_t gx, int32_t gy, int32_t gz, unsigned long long *nodes,
                     void *stream);
/* Every rank's root node emitted once to every other rank (numRanks - 1
 * emits per rank) into the node context. */
rf_status rf_mp_broadcast(rf_ctx *nodeCtx, const unsigned long long *nodes, void *stream);
/* For every incoming root at rank r from a non-empty rank s that is one of
 * r's 26 torus neighbours, a request {r, s, 0, 0} emitted to s. */
rf_status rf_mp_request(rf_ctx *nodeCtx, rf_ctx *requestCtx, int32_t gx, int32_t gy, int32_t gz, void *stream);
/* For every incoming request at rank s, its non-empty octant nodes (up to 8
 * emits per request) emitted to the requester. */
rf_status rf_mp_respond(rf_ctx *requestCtx, rf_ctx *nodeCtx, const unsigned long long *nodes, void *stream);
/* One protocol step: migrate, exchange particles, trees, broadcast, exchange
 * nodes, requests, exchange requests, replies, exchange nodes.  delivered
 * (host, 4 words, nullable) = items delivered by the four exchanges.  Waits
 * for the stream. */
rf_status rf_mp_step(rf_ctx *particles, rf_ctx *nodeCtx, rf_ctx *requestCtx, int32_t gx, int32_t gy, int32_t gz,
                     unsigned long long *nodes, void *stream, uint64_t delivered[4]);

#ifdef __cplusplus
}
#endif

#endif /* RAFI_H */
