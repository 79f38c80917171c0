// Graph form of the forwarding loop: the rounds of "work kernel, then the
// exchange" (Sec. 5.1's loop) run inside one CUDA graph whose conditional
// while node repeats them while the exchange reports active items, so no
// round waits for the host; unlike the persistent kernel, each round's
// kernels launch with their own grid shapes and occupancy.
//
//   init kernel       rounds = forwarded = 0; condition = (numActive > 0 and
//                     maxRounds > 0), from the exchange that seeded the queue
//   while (condition) the round's kernels as the caller enqueues them
//                     (captured once), then the control kernel: rounds += 1,
//                     forwarded += numActive, condition = (numActive > 0 and
//                     rounds < maxRounds)
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

rf_status run_graph_loop(rf_ctx *ctx, cudaStream_t s, uint32_t maxRounds,
                         const std::function<rf_status(cudaStream_t)> &round, uint64_t *rounds, uint64_t *forwarded)
{
    if (!ctx->loopState) RF_CUDA(cudaMalloc(&ctx->loopState, 3 * sizeof(unsigned long long)));
    cudaGraph_t graph = nullptr, body = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    const bool timing = ctx->timing;
    const unsigned long long launches0 = g_launches.load();
    unsigned long long bodyLaunches = 0;
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
        e = cudaGraphAddKernelNode(&initNode, graph, nullptr, 0, &kp);
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
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) { fail(e, "cudaStreamCreate"); break; }
        ctx->timing = false;  // event records may not sit inside a conditional body
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
        // launches: the init kernel, then the captured body once per round
        g_launches.store(launches0);
        count_launch(1ull + bodyLaunches * res[0]);
    } while (0);
    ctx->timing = timing;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    return st;
}

}  // namespace rfi
