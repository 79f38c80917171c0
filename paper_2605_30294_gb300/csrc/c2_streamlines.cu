// Streamlines through a brick-partitioned vector field (Sec. 5.4): every
// particle is one 32-byte work item {position, id, steps, hops, set, status};
// the rank that owns the brick holding it advances it with RK4 steps on the
// trilinear field and forwards it (rafi's emitOutgoing) when a step takes it
// into another rank's brick.  The paper's ranks make one step per round and
// forward every particle, to itself when it stays; stepsPerRound = 1
// reproduces that, stepsPerRound = 0 advances a particle until it leaves the
// brick or stops.  Either way a particle's path is the same.
//
// Built with -fmad=false: the RK4 and trilinear arithmetic follows the
// written order, so a partitioned run reproduces the unpartitioned one.
#include "internal.cuh"
#include "rafi_device.cuh"
#include "rounds.cuh"

namespace rfi {
namespace {

constexpr int kBlock = 256;
constexpr int kHalo = 2;

enum : uint32_t { kExited = 1u, kStalled = 2u, kMaxSteps = 3u };

struct C2Params {
    const float *bricks;   // (N/B)^3 bricks of (B + 2*kHalo)^3 x-pairs of 8 floats (32-byte aligned)
    uint4 *out;            // final particle per id (2 x uint4)
    uint64_t outCap;
    int32_t N, B, nb;
    float h;
    uint32_t maxSteps;
    uint32_t stepsPerRound;  // 0: until the particle leaves its brick
};

__device__ __forceinline__ int32_t clampi(int32_t v, int32_t lo, int32_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int32_t owner_of(float px, float py, float pz, int32_t B, int32_t nb)
{
    const int32_t bx = clampi((int32_t)floorf(px / (float)B), 0, nb - 1);
    const int32_t by = clampi((int32_t)floorf(py / (float)B), 0, nb - 1);
    const int32_t bz = clampi((int32_t)floorf(pz / (float)B), 0, nb - 1);
    return bx + nb * (by + nb * bz);
}

// One brick element: the velocities {vx, vy, vz, 0} of voxel x and of voxel
// x + 1, read by one 32-byte load through the read-only path.
__device__ __forceinline__ void ld_pair(const float *p, float4 &a, float4 &b)
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// Trilinear velocity at p from the brick whose halo origin is org (voxel
// centres at v + 0.5, clamp to the grid edge).  Along y and z the two corner
// indices are clamped to the grid, then to the halo; along x the element at
// lo - org holds both corners (make_bricks_kernel clamps them to the grid),
// so the eight corners take four loads.  A stage point stays within a
// quarter voxel of the brick (speed at most 1, h = 0.25), well inside the
// halo, where this equals the unpartitioned trilinear sample.
__device__ __forceinline__ void sample(const float *__restrict__ brick, int32_t N, int32_t S, const int32_t org[3],
                                       const float p[3], float v[3])
{
    int32_t i0[3], i1[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float u = p[a] - 0.5f;
        const float fl = floorf(u);
        f[a] = u - fl;
        const int32_t lo = (int32_t)fl;
        if (a == 0) {
            i0[a] = clampi(lo - org[a], 0, S - 1);
            i1[a] = i0[a];
        } else {
            i0[a] = clampi(clampi(lo, 0, N - 1) - org[a], 0, S - 1);
            i1[a] = clampi(clampi(lo + 1, 0, N - 1) - org[a], 0, S - 1);
        }
    }
    float4 t000, t100, t010, t110, t001, t101, t011, t111;
    ld_pair(brick + (size_t)8 * ((i0[2] * S + i0[1]) * S + i0[0]), t000, t100);
    ld_pair(brick + (size_t)8 * ((i0[2] * S + i1[1]) * S + i0[0]), t010, t110);
    ld_pair(brick + (size_t)8 * ((i1[2] * S + i0[1]) * S + i0[0]), t001, t101);
    ld_pair(brick + (size_t)8 * ((i1[2] * S + i1[1]) * S + i0[0]), t011, t111);
    const float gx = 1.0f - f[0], gy = 1.0f - f[1], gz = 1.0f - f[2];
#define RF_TRI(c, k)                                       \
    {                                                      \
        const float c00 = t000.c * gx + t100.c * f[0];     \
        const float c10 = t010.c * gx + t110.c * f[0];     \
        const float c01 = t001.c * gx + t101.c * f[0];     \
        const float c11 = t011.c * gx + t111.c * f[0];     \
        const float c0 = c00 * gy + c10 * f[1];            \
        const float c1 = c01 * gy + c11 * f[1];            \
        v[k] = c0 * gz + c1 * f[2];                        \
    }
    RF_TRI(x, 0) RF_TRI(y, 1) RF_TRI(z, 2)
#undef RF_TRI
}

// Advance the particle w on `rank`.  Returns the rank to forward it to, or
// -1 when it stopped (status set in w, written to out[id]).
__device__ int32_t c2_advance(const C2Params &P, uint4 (&w)[2], int32_t rank)
{
    const int32_t S = P.B + 2 * kHalo;
    const int32_t bx = rank % P.nb, by = (rank / P.nb) % P.nb, bz = rank / (P.nb * P.nb);
    const int32_t org[3] = {bx * P.B - kHalo, by * P.B - kHalo, bz * P.B - kHalo};
    const float *brick = P.bricks + (size_t)rank * S * S * S * 8;
    float p[3] = {__uint_as_float(w[0].x), __uint_as_float(w[0].y), __uint_as_float(w[0].z)};
    uint32_t steps = w[1].x, hops = w[1].y, status = 0u, taken = 0u;
    int32_t dst = -1;
    const float h = P.h, half = P.h * 0.5f, sixth = P.h / 6.0f;
    const float fN = (float)P.N;
    for (;;) {
        if (steps >= P.maxSteps) {
            status = kMaxSteps;
            break;
        }
        if (P.stepsPerRound && taken >= P.stepsPerRound) {
            dst = rank;  // the paper's pattern: forwarded to itself after a step
            break;
        }
        float k1[3], k2[3], k3[3], k4[3], t[3], q[3];
        sample(brick, P.N, S, org, p, k1);
#pragma unroll
        for (int a = 0; a < 3; ++a) t[a] = p[a] + half * k1[a];
        sample(brick, P.N, S, org, t, k2);
#pragma unroll
        for (int a = 0; a < 3; ++a) t[a] = p[a] + half * k2[a];
        sample(brick, P.N, S, org, t, k3);
#pragma unroll
        for (int a = 0; a < 3; ++a) t[a] = p[a] + h * k3[a];
        sample(brick, P.N, S, org, t, k4);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float s = ((k1[a] + 2.0f * k2[a]) + 2.0f * k3[a]) + k4[a];
            q[a] = p[a] + sixth * s;
        }
        if (q[0] == p[0] && q[1] == p[1] && q[2] == p[2]) {
            status = kStalled;
            break;
        }
        ++steps;
        ++taken;
        p[0] = q[0];
        p[1] = q[1];
        p[2] = q[2];
        if (!(p[0] >= 0.0f && p[0] < fN && p[1] >= 0.0f && p[1] < fN && p[2] >= 0.0f && p[2] < fN)) {
            status = kExited;
            break;
        }
        const int32_t own = owner_of(p[0], p[1], p[2], P.B, P.nb);
        if (own != rank) {
            ++hops;
            dst = own;
            break;
        }
    }
    w[0].x = __float_as_uint(p[0]);
    w[0].y = __float_as_uint(p[1]);
    w[0].z = __float_as_uint(p[2]);
    w[1].x = steps;
    w[1].y = hops;
    w[1].w = status;
    return dst;
}

__device__ __forceinline__ void c2_write_out(const C2Params &P, const uint4 (&w)[2])
{
    const uint32_t id = w[0].w;
    if (id < P.outCap) {
        P.out[(size_t)id * 2] = w[0];
        P.out[(size_t)id * 2 + 1] = w[1];
    }
}

// The streamline step as a policy of the persistent round kernel.
struct C2Work {
    static constexpr int V = 2;
    static constexpr bool kAppendRetired = false;
    static constexpr bool kDynamicWork = true;
    static constexpr bool kGridStride = false;
    static constexpr bool kFuseStep = false;
    static constexpr unsigned kStepReadMask = 0x3u;  // every vector
    static constexpr unsigned kStepWriteMask = 0x3u;
    static constexpr int kMinBlocksPerSM = 3;
    static constexpr int kItemsPerThread = 1;
    static constexpr int kBlock = kRoundsBlock;
    C2Params P;
    __host__ __device__ uint32_t smemBytes() const { return 0u; }
    __device__ void load_smem(void *) const {}
    __device__ int32_t step(uint4 (&w)[2], int32_t rank, uint32_t, const void *) const
    {
        return c2_advance(P, w, rank);
    }
    __device__ void retire(const uint4 (&w)[2]) const { c2_write_out(P, w); }
};

// Shapes of the persistent kernel for this policy (the autotuner's
// candidates): {items per thread, CTAs per SM, threads}.  The work phase's
// occupancy is what matters here; the tile only sizes the scatter.
using C2Shapes = ShapeList<C2Work, Shape<C2Work, 1, 3, 256>, Shape<C2Work, 1, 2, 256>, Shape<C2Work, 1, 6, 128>,
                           Shape<C2Work, 2, 3, 256>>;


// Element (lx, ly, lz) of brick r holds the grid voxels (gx, gy, gz) and
// (gx + 1, gy, gz) of its halo origin + (lx, ly, lz), each clamped to the grid.
__global__ void __launch_bounds__(kBlock) make_bricks_kernel(const float *__restrict__ field, int32_t N, int32_t B,
                                                             float4 *__restrict__ bricks)
{
    const int32_t nb = N / B, S = B + 2 * kHalo;
    const uint64_t per = (uint64_t)S * S * S;
    const uint64_t total = per * nb * nb * nb;
    for (uint64_t v = blockIdx.x * (uint64_t)kBlock + threadIdx.x; v < total; v += (uint64_t)gridDim.x * kBlock) {
        const int32_t r = (int32_t)(v / per);
        const int32_t l = (int32_t)(v % per);
        const int32_t lx = l % S, ly = (l / S) % S, lz = l / (S * S);
        const int32_t bx = r % nb, by = (r / nb) % nb, bz = r / (nb * nb);
        const int32_t gx = clampi(bx * B - kHalo + lx, 0, N - 1);
        const int32_t gx1 = clampi(bx * B - kHalo + lx + 1, 0, N - 1);
        const int32_t gy = clampi(by * B - kHalo + ly, 0, N - 1);
        const int32_t gz = clampi(bz * B - kHalo + lz, 0, N - 1);
        const float *row = field + ((size_t)gz * N + gy) * N * 3u;
        const float *f = row + (size_t)gx * 3u, *f1 = row + (size_t)gx1 * 3u;
        bricks[2 * v] = make_float4(f[0], f[1], f[2], 0.0f);
        bricks[2 * v + 1] = make_float4(f1[0], f1[1], f1[2], 0.0f);
    }
}

// Seed: particle i at seeds[i] with id i and set setIds[i] (or 0) is
// emitted, in out slot i, to the rank owning its position.
__global__ void __launch_bounds__(kBlock) seed_kernel(const float *__restrict__ seeds,
                                                      const uint32_t *__restrict__ setIds, uint32_t n, int32_t B,
                                                      int32_t nb, rf_device_queues q)
{
    uint4 *outq = static_cast<uint4 *>(q.out);
    for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        const float x = seeds[3 * (size_t)i], y = seeds[3 * (size_t)i + 1], z = seeds[3 * (size_t)i + 2];
        outq[(size_t)i * 2] = make_uint4(__float_as_uint(x), __float_as_uint(y), __float_as_uint(z), i);
        outq[(size_t)i * 2 + 1] = make_uint4(0u, 0u, setIds ? setIds[i] : 0u, 0u);
        q.dest[i] = owner_of(x, y, z, B, nb);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *q.outCount = n;
}

// Plain per-rank trace kernel of one round: incoming particle i advances on
// its rank; out slot i holds it when forwarded, destination -1 when it stopped.
__global__ void __launch_bounds__(kBlock) trace_kernel(C2Params P, rf_device_queues q)
{
    __shared__ uint32_t sOff[RF_MAX_RANKS + 1];
    const int32_t R = q.numRanks;
    for (int e = threadIdx.x; e <= R; e += kBlock) sOff[e] = q.inOffset[e];
    __syncthreads();
    const uint32_t n = sOff[R];
    if (blockIdx.x == 0 && threadIdx.x == 0) *q.outCount = n;
    const uint4 *inq = static_cast<const uint4 *>(q.in);
    uint4 *outq = static_cast<uint4 *>(q.out);
    for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        uint4 w[2] = {__ldg(inq + (size_t)i * 2), __ldg(inq + (size_t)i * 2 + 1)};
        const int32_t rank = rf::rankOf(sOff, R, i);
        const int32_t d = c2_advance(P, w, rank);
        if (d >= 0) {
            outq[(size_t)i * 2] = w[0];
            outq[(size_t)i * 2 + 1] = w[1];
        } else {
            c2_write_out(P, w);
        }
        q.dest[i] = d;
    }
}

rf_status check_c2(rf_ctx *ctx, int32_t N, int32_t B, const char *fn)
{
    if (!ctx) {
        set_error("%s: NULL context", fn);
        return RF_ERR_ARG;
    }
    if (ctx->itemBytes != 32) {
        set_error("%s: particles are 32 bytes (context has %u)", fn, ctx->itemBytes);
        return RF_ERR_ARG;
    }
    if (N < 1 || B < 1 || N % B || (int64_t)(N / B) * (N / B) * (N / B) != ctx->numRanks) {
        set_error("%s: N %d, brick %d do not give %d ranks", fn, N, B, ctx->numRanks);
        return RF_ERR_ARG;
    }
    return RF_OK;
}

C2Params make_params(const float *bricks, int32_t N, int32_t B, float h, uint32_t maxSteps, uint32_t stepsPerRound,
                     void *out, uint64_t outCap)
{
    C2Params P;
    P.bricks = bricks;
    P.out = static_cast<uint4 *>(out);
    P.outCap = outCap;
    P.N = N;
    P.B = B;
    P.nb = N / B;
    P.h = h;
    P.maxSteps = maxSteps;
    P.stepsPerRound = stepsPerRound;
    return P;
}

int grid_for(rf_ctx *ctx, uint64_t work)
{
    const uint64_t want = (work + kBlock - 1) / kBlock;
    const uint64_t cap = (uint64_t)ctx->numSMs * 8u;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace
}  // namespace rfi

using namespace rfi;

namespace rfi {
int c2_shapes(int32_t *out, int32_t cap)
{
    ShapeInfo v[C2Shapes::kCount];
    C2Shapes::infos(v);
    for (int i = 0; i < C2Shapes::kCount && i < cap; ++i) {
        out[3 * i] = v[i].block;
        out[3 * i + 1] = v[i].itemsPerThread;
        out[3 * i + 2] = v[i].ctasPerSM;
    }
    return C2Shapes::kCount;
}
}  // namespace rfi

extern "C" {

rf_status rf_c2_make_bricks(const float *field, int32_t N, int32_t B, float *bricks, void *stream)
{
    if (!field || !bricks || N < 1 || B < 1 || N % B || (reinterpret_cast<uintptr_t>(bricks) & 31u)) {
        set_error("rf_c2_make_bricks: bad arguments (bricks must be 32-byte aligned)");
        return RF_ERR_ARG;
    }
    const int32_t nb = N / B, S = B + 2 * kHalo;
    const uint64_t total = (uint64_t)S * S * S * nb * nb * nb;
    uint64_t blocks = (total + kBlock - 1) / kBlock;
    if (blocks > 65535u * 16u) blocks = 65535u * 16u;
    make_bricks_kernel<<<(unsigned)blocks, kBlock, 0, static_cast<cudaStream_t>(stream)>>>(
        field, N, B, reinterpret_cast<float4 *>(bricks));
    RF_LAUNCHED("c2 make_bricks_kernel");
    return RF_OK;
}

rf_status rf_c2_seed(rf_ctx *ctx, const float *seeds, const uint32_t *setIds, uint64_t n, int32_t N, int32_t B,
                     void *stream)
{
    if (rf_status st = check_c2(ctx, N, B, "rf_c2_seed")) return st;
    if (n > ctx->capacity || (n && !seeds)) {
        set_error("rf_c2_seed: n %llu above capacity or NULL seeds", (unsigned long long)n);
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    rf_device_queues q;
    rf_get_device_queues(ctx, &q);
    seed_kernel<<<grid_for(ctx, n), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(seeds, setIds, (uint32_t)n, B,
                                                                                    N / B, q);
    RF_LAUNCHED("c2 seed_kernel");
    return RF_OK;
}

rf_status rf_c2_trace(rf_ctx *ctx, const float *bricks, int32_t N, int32_t B, float h, uint32_t maxSteps,
                      uint32_t stepsPerRound, void *out, uint64_t outCapacity, void *stream)
{
    if (rf_status st = check_c2(ctx, N, B, "rf_c2_trace")) return st;
    if (!bricks || !out || !(h > 0.0f) || (reinterpret_cast<uintptr_t>(bricks) & 31u)) {
        set_error("rf_c2_trace: NULL or unaligned bricks, NULL out or step <= 0");
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    rf_device_queues q;
    rf_get_device_queues(ctx, &q);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const C2Params P = make_params(bricks, N, B, h, maxSteps, stepsPerRound, out, outCapacity);
    time_begin(ctx, kTimeWork, s);
    trace_kernel<<<grid_for(ctx, ctx->capacity), kBlock, 0, s>>>(P, q);
    RF_LAUNCHED("c2 trace_kernel");
    time_end(ctx, kTimeWork, s);
    return RF_OK;
}

rf_status rf_c2_run(rf_ctx *ctx, const float *bricks, const float *seeds, const uint32_t *setIds, uint64_t n,
                    int32_t N, int32_t B, float h, uint32_t maxSteps, uint32_t stepsPerRound, void *out,
                    int32_t batched, uint32_t maxRounds, void *stream, uint64_t *rounds, uint64_t *forwarded)
{
    if (rf_status st = check_c2(ctx, N, B, "rf_c2_run")) return st;
    if (!bricks || !out || (n && !seeds) || n > ctx->capacity || !(h > 0.0f) ||
        (reinterpret_cast<uintptr_t>(bricks) & 31u) || batched < RF_FORM_HOST_LOOP || batched > RF_FORM_TUNED) {
        set_error("rf_c2_run: bad arguments");
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (rf_status st = rf_c2_seed(ctx, seeds, setIds, n, N, B, stream)) return st;
    const C2Params P = make_params(bricks, N, B, h, maxSteps, stepsPerRound, out, n);
    // RF_FORM_TUNED: the form the context holds for this policy (set by the autotuner)
    const int32_t form = batched == RF_FORM_TUNED ? ctx->batchedForm[RF_POLICY_STREAMLINES] : batched;
    uint64_t active = 0, fwd = 0, r = 0;
    if (form == RF_FORM_GRAPH) {
        // graph form: the trace kernel and the exchange repeated by a while node
        if (rf_status st = rf_exchange(ctx, stream, nullptr)) return st;
        rf_status st = run_graph_loop(ctx, s, maxRounds, [&](cudaStream_t cs) -> rf_status {
            rf_device_queues q;
            rf_get_device_queues(ctx, &q);
            trace_kernel<<<grid_for(ctx, ctx->capacity), kBlock, 0, cs>>>(P, q);
            RF_LAUNCHED("c2 trace_kernel");
            return launch_exchange(ctx, cs);
        }, &r, &fwd);
        if (st != RF_OK) return st;
        active = ctx->host->numActive;
    } else if (form == RF_FORM_PERSISTENT) {
        if (rf_status st = rf_exchange(ctx, stream, nullptr)) return st;
        C2Work w;
        w.P = P;
        unsigned long long res[4];
        rf_status st = C2Shapes::launch(ctx->batchedShape[RF_POLICY_STREAMLINES], ctx, w, maxRounds, s, nullptr,
                                        0u, nullptr, 0ull, nullptr, res);
        if (st != RF_OK) return st;
        r = res[0];
        fwd = res[1];
        active = ctx->host->numActive;
    } else {
        rf_status st = rf_exchange(ctx, stream, &active);
        if (st != RF_OK) return st;
        while (active > 0 && r < maxRounds) {
            if ((st = rf_c2_trace(ctx, bricks, N, B, h, maxSteps, stepsPerRound, out, n, stream))) return st;
            if ((st = rf_exchange(ctx, stream, &active))) return st;
            fwd += active;
            ++r;
        }
    }
    if (rounds) *rounds = r;
    if (forwarded) *forwarded = fwd;
    if (active) {
        set_error("rf_c2_run: %llu particles still active after %u rounds", (unsigned long long)active, maxRounds);
        return RF_ERR_MAX_ROUNDS;
    }
    return RF_OK;
}

}  // extern "C"
