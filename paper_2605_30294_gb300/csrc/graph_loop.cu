// Graph form of the forwarding loop: the rounds of "work kernel, then the
// exchange" (Sec. 5.1's loop) run inside one CUDA graph whose conditional
// while node repeats them while the exchange reports active items, so no
// round waits for the host; unlike the persistent kernel, each round's
// kernels launch with their own grid shapes and occupancy.
//
//   prologue          (optional, a child graph) the kernels that seed the
//                     queue and its first exchange
//   init kernel       rounds = forwarded = 0; condition = (numActive > 0 and
//                     maxRounds > 0), from the exchange that seeded the queue
//   while (condition) the round's kernels as the caller enqueues them
//                     (captured once), then the control kernel: rounds += 1,
//                     forwarded += numActive, condition = (numActive > 0 and
//                     rounds < maxRounds)
//
// A caller that passes a key keeps the instantiated graph in the context and
// relaunches it while the key (every pointer and value its kernels take)
// stays the same; the context holds one such graph at a time.
#include <functional>

#include "internal.cuh"

namespace rfi {
namespace {

// loop state on the device: {rounds, forwarded, maxRounds}
__global__ void loop_init_kernel(cudaGraphConditionalHandle h, const DevState *st, unsigned long long *ls,
                                 unsigned long long maxRounds)
{
    if (threadIdx.x == 0) {
        ls[0] = 0ull;
        ls[1] = 0ull;
        ls[2] = maxRounds;
        cudaGraphSetConditional(h, (st->numActive > 0ull && maxRounds > 0ull) ? 1u : 0u);
    }
}

__global__ void loop_control_kernel(cudaGraphConditionalHandle h, const DevState *st, unsigned long long *ls)
{
    if (threadIdx.x == 0) {
        const unsigned long long r = ls[0] + 1ull;
        ls[0] = r;
        ls[1] += st->numActive;
        cudaGraphSetConditional(h, (st->numActive > 0ull && r < ls[2]) ? 1u : 0u);
    }
}

}  // namespace

void drop_graph_loop(rf_ctx *ctx)
{
    if (ctx->loopExec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(ctx->loopExec));
    if (ctx->loopGraph) cudaGraphDestroy(static_cast<cudaGraph_t>(ctx->loopGraph));
    ctx->loopExec = nullptr;
    ctx->loopGraph = nullptr;
    ctx->loopKey.clear();
    ctx->loopLaunchesPerRound = 0;
    ctx->loopLaunchesOnce = 0;
}

rf_status run_graph_loop(rf_ctx *ctx, cudaStream_t s, uint32_t maxRounds,
                         const std::function<rf_status(cudaStream_t)> &round, uint64_t *rounds, uint64_t *forwarded,
                         const std::function<rf_status(cudaStream_t)> &prologue, const void *key, size_t keyBytes)
{
    if (!ctx->loopState) RF_CUDA(cudaMalloc(&ctx->loopState, 3 * sizeof(unsigned long long)));
    std::string k;
    if (key) {
        // the caller's key, the round limit and the exchange's launch shape
        const uint64_t shape[4] = {maxRounds, ctx->tileItems, (uint64_t)ctx->scatterBlocks,
                                   (uint64_t)ctx->countBlocks};
        k.assign(static_cast<const char *>(key), keyBytes);
        k.append(reinterpret_cast<const char *>(shape), sizeof shape);
    }
    const unsigned long long launches0 = g_launches.load();
    if (key && ctx->loopExec && ctx->loopKey == k) {
        // the same loop as last time: relaunch the instantiated graph
        RF_CUDA(cudaGraphLaunch(static_cast<cudaGraphExec_t>(ctx->loopExec), s));
        unsigned long long res[3] = {0, 0, 0};
        RF_CUDA(cudaMemcpyAsync(res, ctx->loopState, sizeof res, cudaMemcpyDeviceToHost, s));
        RF_CUDA(cudaMemcpyAsync(ctx->host, ctx->dev, sizeof(DevState), cudaMemcpyDeviceToHost, s));
        RF_CUDA(cudaStreamSynchronize(s));
        ctx->pending = false;
        if (rounds) *rounds = res[0];
        if (forwarded) *forwarded = res[1];
        count_launch(ctx->loopLaunchesOnce + ctx->loopLaunchesPerRound * res[0]);
        return RF_OK;
    }
    drop_graph_loop(ctx);
    cudaGraph_t graph = nullptr, body = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    const bool timing = ctx->timing;
    unsigned long long bodyLaunches = 0, onceLaunches = 1;
    rf_status st = RF_OK;
    auto fail = [&](cudaError_t e, const char *what) {
        st = cuda_fail(e, what);
        return st;
    };
    do {
        cudaError_t e = cudaGraphCreate(&graph, 0);
        if (e != cudaSuccess) { fail(e, "cudaGraphCreate"); break; }
        cudaGraphConditionalHandle h;
        e = cudaGraphConditionalHandleCreate(&h, graph, 0u, 0u);
        if (e != cudaSuccess) { fail(e, "cudaGraphConditionalHandleCreate"); break; }
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) { fail(e, "cudaStreamCreate"); break; }
        ctx->timing = false;  // event records may not sit inside a conditional body
        // the prologue, captured into a child graph
        cudaGraphNode_t proNode = nullptr;
        if (prologue) {
            cudaGraph_t pro = nullptr;
            e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
            if (e != cudaSuccess) { fail(e, "cudaStreamBeginCapture"); break; }
            const unsigned long long p0 = g_launches.load();
            rf_status ps = prologue(cap);
            onceLaunches += g_launches.load() - p0;
            e = cudaStreamEndCapture(cap, &pro);
            if (ps != RF_OK) { st = ps; if (pro) cudaGraphDestroy(pro); break; }
            if (e != cudaSuccess) { fail(e, "cudaStreamEndCapture(prologue)"); break; }
            e = cudaGraphAddChildGraphNode(&proNode, graph, nullptr, 0, pro);
            cudaGraphDestroy(pro);  // the node holds its own copy
            if (e != cudaSuccess) { fail(e, "cudaGraphAddChildGraphNode"); break; }
        }
        // init kernel node
        cudaKernelNodeParams kp = {};
        const DevState *stp = ctx->dev;
        unsigned long long *ls = static_cast<unsigned long long *>(ctx->loopState);
        unsigned long long maxR = maxRounds;
        void *initArgs[] = {&h, &stp, &ls, &maxR};
        kp.func = reinterpret_cast<void *>(loop_init_kernel);
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32);
        kp.kernelParams = initArgs;
        cudaGraphNode_t initNode;
        e = cudaGraphAddKernelNode(&initNode, graph, proNode ? &proNode : nullptr, proNode ? 1 : 0, &kp);
        if (e != cudaSuccess) { fail(e, "cudaGraphAddKernelNode(init)"); break; }
        // conditional while node after it
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t loopNode;
        e = cudaGraphAddNode(&loopNode, graph, &initNode, nullptr, 1, &cp);
        if (e != cudaSuccess) { fail(e, "cudaGraphAddNode(while)"); break; }
        body = cp.conditional.phGraph_out[0];
        // the round's kernels and the control kernel, captured into the body
        e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) { fail(e, "cudaStreamBeginCaptureToGraph"); break; }
        const unsigned long long c0 = g_launches.load();
        rf_status rs = round(cap);
        if (rs == RF_OK) {
            loop_control_kernel<<<1, 32, 0, cap>>>(h, stp, ls);
            if (cudaGetLastError() != cudaSuccess) rs = RF_ERR_CUDA;
        }
        bodyLaunches = g_launches.load() - c0 + 1;
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(cap, &captured);
        if (rs != RF_OK) { st = rs; break; }
        if (e != cudaSuccess) { fail(e, "cudaStreamEndCapture"); break; }
        e = cudaGraphInstantiate(&exec, graph, 0ull);
        if (e != cudaSuccess) { fail(e, "cudaGraphInstantiate"); break; }
        e = cudaGraphLaunch(exec, s);
        if (e != cudaSuccess) { fail(e, "cudaGraphLaunch"); break; }
        unsigned long long res[3] = {0, 0, 0};
        e = cudaMemcpyAsync(res, ctx->loopState, sizeof res, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) { fail(e, "cudaMemcpyAsync(loop state)"); break; }
        e = cudaMemcpyAsync(ctx->host, ctx->dev, sizeof(DevState), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) { fail(e, "cudaMemcpyAsync(state)"); break; }
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { fail(e, "cudaStreamSynchronize"); break; }
        ctx->pending = false;
        if (rounds) *rounds = res[0];
        if (forwarded) *forwarded = res[1];
        // launches: the prologue and the init kernel, then the body once per round
        g_launches.store(launches0);
        count_launch(onceLaunches + bodyLaunches * res[0]);
        if (key) {
            ctx->loopExec = exec;
            ctx->loopGraph = graph;
            ctx->loopKey = k;
            ctx->loopLaunchesPerRound = bodyLaunches;
            ctx->loopLaunchesOnce = onceLaunches;
            exec = nullptr;
            graph = nullptr;
        }
    } while (0);
    ctx->timing = timing;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    if (st != RF_OK) g_launches.store(launches0);
    return st;
}

}  // namespace rfi
