// Multi-phase exchange with three item types: the communication pattern of
// the paper's distributed Barnes-Hut N-body code (Sec. 5.5), where one
// program drives three forwarding contexts of different item types on one
// stream - particle migration, then an essential-tree exchange in which every
// rank broadcasts its root multipole node, peers that need finer data send a
// refinement request back, and the owner answers with child nodes.
//
// The workload is synthetic and integer-only, so every result is exact:
// positions are 32-bit fixed point on the periodic unit cube, split into a
// gx x gy x gz grid of ranks (powers of two); a node holds the mass, the
// mass-weighted coordinate sums and the particle count of one rank (its root)
// or of one octant of the rank's box (a child).  A peer asks for children
// when it is one of the 26 torus neighbours of the node's rank and the node
// is not empty.  Two of the kernels emit several items per input: the root
// broadcast (numRanks - 1 per rank) and the reply (up to 8 per request).
#include "internal.cuh"
#include "rafi_device.cuh"

namespace rfi {
namespace {

constexpr int kBlock = 256;

struct __align__(16) Particle {
    uint32_t x, y, z;
    int32_t vx, vy, vz;
    uint32_t m, id;
};
static_assert(sizeof(Particle) == 32, "32-byte particle");

struct __align__(16) Node {
    unsigned long long M, X, Y, Z;
    uint32_t count, src, code, level;
    uint32_t pad[4];
};
static_assert(sizeof(Node) == 64, "64-byte node");

struct __align__(16) Request {
    uint32_t requester, target, code, level;
};
static_assert(sizeof(Request) == 16, "16-byte request");

// node accumulators per rank: root, then octants 0..7, 5 words each
constexpr int kNodeWords = 5;
constexpr int kNodesPerRank = 9;

struct Grid {
    int32_t lg[3];
};

__device__ __forceinline__ int32_t owner_of(uint32_t x, uint32_t y, uint32_t z, const Grid &g)
{
    const uint32_t bx = g.lg[0] ? x >> (32 - g.lg[0]) : 0u;
    const uint32_t by = g.lg[1] ? y >> (32 - g.lg[1]) : 0u;
    const uint32_t bz = g.lg[2] ? z >> (32 - g.lg[2]) : 0u;
    return (int32_t)(bx + (by << g.lg[0]) + (bz << (g.lg[0] + g.lg[1])));
}

__device__ __forceinline__ int32_t octant_of(uint32_t x, uint32_t y, uint32_t z, const Grid &g)
{
    return (int32_t)(((x >> (31 - g.lg[0])) & 1u) | (((y >> (31 - g.lg[1])) & 1u) << 1) |
                     (((z >> (31 - g.lg[2])) & 1u) << 2));
}

// one of the 26 torus neighbours (per-axis wrapped distance at most 1, not equal)
__device__ __forceinline__ bool near_ranks(int32_t r, int32_t s, const Grid &g)
{
    if (r == s) return false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int32_t side = 1 << g.lg[k];
        const int32_t shift = k == 0 ? 0 : (k == 1 ? g.lg[0] : g.lg[0] + g.lg[1]);
        const int32_t a = (r >> shift) & (side - 1), b = (s >> shift) & (side - 1);
        const int32_t d = (a - b + side) & (side - 1);
        if (d != 0 && d != 1 && d != side - 1) return false;
    }
    return true;
}

__global__ void __launch_bounds__(kBlock) seed_kernel(const Particle *p, uint32_t n, rf_device_queues q, Grid g)
{
    for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        const Particle a = p[i];
        rf::forward(q, a, owner_of(a.x, a.y, a.z, g));
    }
}

// Migration (Sec. 5.5): each particle moves by its velocity, wrapping around
// the cube, and is forwarded to the rank that owns its new position.
__global__ void __launch_bounds__(kBlock) migrate_kernel(rf_device_queues q, Grid g)
{
    const uint32_t n = rf::numIncoming(q);
    for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        Particle a = rf::getIncoming<Particle>(q, i);
        a.x += (uint32_t)a.vx;
        a.y += (uint32_t)a.vy;
        a.z += (uint32_t)a.vz;
        rf::forward(q, a, owner_of(a.x, a.y, a.z, g));
    }
}

// Local trees: CTA r reduces rank r's incoming particles into its root and
// eight octant nodes (shared-memory 64-bit atomics, exact).
__global__ void __launch_bounds__(kBlock) tree_kernel(rf_device_queues q, Grid g, unsigned long long *nodes)
{
    __shared__ unsigned long long acc[kNodesPerRank * kNodeWords];
    const int32_t r = blockIdx.x;
    for (int e = threadIdx.x; e < kNodesPerRank * kNodeWords; e += kBlock) acc[e] = 0ull;
    __syncthreads();
    const uint32_t lo = q.inOffset[r], hi = q.inOffset[r + 1];
    for (uint32_t i = lo + threadIdx.x; i < hi; i += kBlock) {
        const Particle a = rf::getIncoming<Particle>(q, i);
        const int c[2] = {0, 1 + octant_of(a.x, a.y, a.z, g)};
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            unsigned long long *nd = acc + c[j] * kNodeWords;
            atomicAdd(&nd[0], (unsigned long long)a.m);
            atomicAdd(&nd[1], (unsigned long long)a.m * a.x);
            atomicAdd(&nd[2], (unsigned long long)a.m * a.y);
            atomicAdd(&nd[3], (unsigned long long)a.m * a.z);
            atomicAdd(&nd[4], 1ull);
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kNodesPerRank * kNodeWords; e += kBlock)
        nodes[(size_t)r * kNodesPerRank * kNodeWords + e] = acc[e];
}

__device__ __forceinline__ Node make_node(const unsigned long long *nd, int32_t src, uint32_t code)
{
    Node v;
    v.M = nd[0];
    v.X = nd[1];
    v.Y = nd[2];
    v.Z = nd[3];
    v.count = (uint32_t)nd[4];
    v.src = (uint32_t)src;
    v.code = code;
    v.level = code == 0u ? 0u : 1u;
#pragma unroll
    for (int k = 0; k < 4; ++k) v.pad[k] = 0u;
    return v;
}

// Root broadcast: CTA s emits its root node once to every other rank.
__global__ void __launch_bounds__(kBlock) broadcast_kernel(rf_device_queues q, const unsigned long long *nodes)
{
    const int32_t s = blockIdx.x;
    const Node v = make_node(nodes + (size_t)s * kNodesPerRank * kNodeWords, s, 0u);
    for (int32_t r = threadIdx.x; r < q.numRanks; r += kBlock)
        if (r != s) rf::forward(q, v, r);
}

// Refinement requests: a root that arrived at rank r from a near, non-empty
// rank s makes r ask s for its children (read from the node context's
// incoming queue, emitted into the request context).
__global__ void __launch_bounds__(kBlock) request_kernel(rf_device_queues nq, rf_device_queues rq, Grid g)
{
    const uint32_t n = rf::numIncoming(nq);
    for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        const Node v = rf::getIncoming<Node>(nq, i);
        const int32_t r = rf::rankOf(nq, i);
        const int32_t s = (int32_t)v.src;
        if (v.code == 0u && v.count > 0u && near_ranks(r, s, g)) {
            Request req;
            req.requester = (uint32_t)r;
            req.target = (uint32_t)s;
            req.code = v.code;
            req.level = v.level;
            rf::forward(rq, req, s);
        }
    }
}

// Replies: rank s answers each request with its non-empty octant nodes.
__global__ void __launch_bounds__(kBlock) respond_kernel(rf_device_queues rq, rf_device_queues nq,
                                                         const unsigned long long *nodes)
{
    const uint32_t n = rf::numIncoming(rq);
    for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        const Request req = rf::getIncoming<Request>(rq, i);
        const int32_t s = rf::rankOf(rq, i);
        const unsigned long long *nd = nodes + (size_t)s * kNodesPerRank * kNodeWords;
        for (int o = 0; o < 8; ++o) {
            const unsigned long long *c = nd + (1 + o) * kNodeWords;
            if (c[4] > 0ull) rf::forward(nq, make_node(c, s, 1u + (uint32_t)o), (int32_t)req.requester);
        }
    }
}

int grid_blocks(const rf_ctx *ctx) { return ctx->numSMs * 8; }

rf_status grid_of(int32_t gx, int32_t gy, int32_t gz, int32_t numRanks, Grid &g, const char *fn)
{
    const int32_t side[3] = {gx, gy, gz};
    for (int k = 0; k < 3; ++k) {
        if (side[k] < 1 || side[k] > (1 << 10) || (side[k] & (side[k] - 1))) {
            set_error("%s: grid sides must be powers of two up to 1024, got %dx%dx%d", fn, gx, gy, gz);
            return RF_ERR_ARG;
        }
        g.lg[k] = 31 - __builtin_clz((unsigned)side[k]);
    }
    if ((long long)gx * gy * gz != numRanks) {
        set_error("%s: grid %dx%dx%d does not have %d ranks", fn, gx, gy, gz, numRanks);
        return RF_ERR_ARG;
    }
    return RF_OK;
}

rf_status check_ctx(const rf_ctx *ctx, uint32_t itemBytes, const char *what, const char *fn)
{
    if (!ctx) {
        set_error("%s: NULL %s context", fn, what);
        return RF_ERR_ARG;
    }
    if (ctx->itemBytes != itemBytes) {
        set_error("%s: the %s context moves %u-byte items, not %u", fn, what, ctx->itemBytes, itemBytes);
        return RF_ERR_ARG;
    }
    return RF_OK;
}

rf_status check_pair(const rf_ctx *a, const rf_ctx *b, const char *fn)
{
    if (a->numRanks != b->numRanks || a->device != b->device) {
        set_error("%s: the contexts differ in rank count or device", fn);
        return RF_ERR_ARG;
    }
    return RF_OK;
}

}  // namespace
}  // namespace rfi

using namespace rfi;

extern "C" rf_status rf_mp_seed(rf_ctx *particles, const void *items, uint64_t n, int32_t gx, int32_t gy, int32_t gz,
                                void *stream)
{
    if (rf_status st = check_ctx(particles, 32u, "particle", "rf_mp_seed")) return st;
    Grid g;
    if (rf_status st = grid_of(gx, gy, gz, particles->numRanks, g, "rf_mp_seed")) return st;
    if (n > 0xFFFFFFFFull || (n && !items)) {
        set_error("rf_mp_seed: NULL items or more than 2^32 - 1 of them");
        return RF_ERR_ARG;
    }
    DeviceGuard dg(particles->device);
    if (!n) return RF_OK;
    rf_device_queues q;
    rf_get_device_queues(particles, &q);
    seed_kernel<<<grid_blocks(particles), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const Particle *>(items), (uint32_t)n, q, g);
    RF_LAUNCHED("multiphase seed_kernel");
    return RF_OK;
}

extern "C" rf_status rf_mp_migrate(rf_ctx *particles, int32_t gx, int32_t gy, int32_t gz, void *stream)
{
    if (rf_status st = check_ctx(particles, 32u, "particle", "rf_mp_migrate")) return st;
    Grid g;
    if (rf_status st = grid_of(gx, gy, gz, particles->numRanks, g, "rf_mp_migrate")) return st;
    DeviceGuard dg(particles->device);
    rf_device_queues q;
    rf_get_device_queues(particles, &q);
    migrate_kernel<<<grid_blocks(particles), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(q, g);
    RF_LAUNCHED("multiphase migrate_kernel");
    return RF_OK;
}

extern "C" rf_status rf_mp_tree(rf_ctx *particles, int32_t gx, int32_t gy, int32_t gz, unsigned long long *nodes,
                                void *stream)
{
    if (rf_status st = check_ctx(particles, 32u, "particle", "rf_mp_tree")) return st;
    Grid g;
    if (rf_status st = grid_of(gx, gy, gz, particles->numRanks, g, "rf_mp_tree")) return st;
    if (!nodes) {
        set_error("rf_mp_tree: NULL nodes");
        return RF_ERR_ARG;
    }
    DeviceGuard dg(particles->device);
    rf_device_queues q;
    rf_get_device_queues(particles, &q);
    tree_kernel<<<particles->numRanks, kBlock, 0, static_cast<cudaStream_t>(stream)>>>(q, g, nodes);
    RF_LAUNCHED("multiphase tree_kernel");
    return RF_OK;
}

extern "C" rf_status rf_mp_broadcast(rf_ctx *nodeCtx, const unsigned long long *nodes, void *stream)
{
    if (rf_status st = check_ctx(nodeCtx, 64u, "node", "rf_mp_broadcast")) return st;
    if (!nodes) {
        set_error("rf_mp_broadcast: NULL nodes");
        return RF_ERR_ARG;
    }
    DeviceGuard dg(nodeCtx->device);
    rf_device_queues q;
    rf_get_device_queues(nodeCtx, &q);
    broadcast_kernel<<<nodeCtx->numRanks, kBlock, 0, static_cast<cudaStream_t>(stream)>>>(q, nodes);
    RF_LAUNCHED("multiphase broadcast_kernel");
    return RF_OK;
}

extern "C" rf_status rf_mp_request(rf_ctx *nodeCtx, rf_ctx *requestCtx, int32_t gx, int32_t gy, int32_t gz,
                                   void *stream)
{
    if (rf_status st = check_ctx(nodeCtx, 64u, "node", "rf_mp_request")) return st;
    if (rf_status st = check_ctx(requestCtx, 16u, "request", "rf_mp_request")) return st;
    if (rf_status st = check_pair(nodeCtx, requestCtx, "rf_mp_request")) return st;
    Grid g;
    if (rf_status st = grid_of(gx, gy, gz, nodeCtx->numRanks, g, "rf_mp_request")) return st;
    DeviceGuard dg(nodeCtx->device);
    rf_device_queues nq, rq;
    rf_get_device_queues(nodeCtx, &nq);
    rf_get_device_queues(requestCtx, &rq);
    request_kernel<<<grid_blocks(nodeCtx), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(nq, rq, g);
    RF_LAUNCHED("multiphase request_kernel");
    return RF_OK;
}

extern "C" rf_status rf_mp_respond(rf_ctx *requestCtx, rf_ctx *nodeCtx, const unsigned long long *nodes,
                                   void *stream)
{
    if (rf_status st = check_ctx(nodeCtx, 64u, "node", "rf_mp_respond")) return st;
    if (rf_status st = check_ctx(requestCtx, 16u, "request", "rf_mp_respond")) return st;
    if (rf_status st = check_pair(nodeCtx, requestCtx, "rf_mp_respond")) return st;
    if (!nodes) {
        set_error("rf_mp_respond: NULL nodes");
        return RF_ERR_ARG;
    }
    DeviceGuard dg(nodeCtx->device);
    rf_device_queues nq, rq;
    rf_get_device_queues(nodeCtx, &nq);
    rf_get_device_queues(requestCtx, &rq);
    respond_kernel<<<grid_blocks(requestCtx), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(rq, nq, nodes);
    RF_LAUNCHED("multiphase respond_kernel");
    return RF_OK;
}

extern "C" rf_status rf_mp_step(rf_ctx *particles, rf_ctx *nodeCtx, rf_ctx *requestCtx, int32_t gx, int32_t gy,
                                int32_t gz, unsigned long long *nodes, void *stream, uint64_t delivered[4])
{
    if (rf_status st = check_ctx(particles, 32u, "particle", "rf_mp_step")) return st;
    if (rf_status st = check_ctx(nodeCtx, 64u, "node", "rf_mp_step")) return st;
    if (rf_status st = check_ctx(requestCtx, 16u, "request", "rf_mp_step")) return st;
    if (rf_status st = check_pair(particles, nodeCtx, "rf_mp_step")) return st;
    if (rf_status st = check_pair(nodeCtx, requestCtx, "rf_mp_step")) return st;
    uint64_t got[4] = {0, 0, 0, 0};
    if (rf_status st = rf_mp_migrate(particles, gx, gy, gz, stream)) return st;
    if (rf_status st = rf_exchange(particles, stream, &got[0])) return st;
    if (rf_status st = rf_mp_tree(particles, gx, gy, gz, nodes, stream)) return st;
    if (rf_status st = rf_mp_broadcast(nodeCtx, nodes, stream)) return st;
    if (rf_status st = rf_exchange(nodeCtx, stream, &got[1])) return st;
    if (rf_status st = rf_mp_request(nodeCtx, requestCtx, gx, gy, gz, stream)) return st;
    if (rf_status st = rf_exchange(requestCtx, stream, &got[2])) return st;
    if (rf_status st = rf_mp_respond(requestCtx, nodeCtx, nodes, stream)) return st;
    if (rf_status st = rf_exchange(nodeCtx, stream, &got[3])) return st;
    if (delivered)
        for (int k = 0; k < 4; ++k) delivered[k] = got[k];
    return RF_OK;
}
