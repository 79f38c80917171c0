// Stochastic transport by delta tracking through a brick-partitioned
// extinction grid: VoPaT's trace step (Sec. 5.1, Fig. 1) - a ray that
// collides scatters and stays (forwarded to its own rank), a ray whose next
// tentative collision lies in another rank's brick is forwarded there, a ray
// that leaves the grid scores the environment radiance.
//
// Every random number is Philox4x32-10 keyed by (pixel, sample, bounce,
// event index), and the event index travels with the ray, so forwarding
// never changes a path.  A ray forwarded at a tentative collision point
// carries that point ("pending"): the receiving rank redraws the same event
// and resolves it with its own brick.
//
// Built with -fmad=false (the written float order, as the oracle's).
#include "internal.cuh"
#include "philox.cuh"
#include "rafi_device.cuh"
#include "rounds.cuh"

namespace rfi {
namespace {

constexpr int kBlock = 256;

// 64-byte path state
struct __align__(16) TRay {
    float px, py, pz, dx;
    float dy, dz;
    uint32_t bounce, event;
    uint32_t gpix, sample, pending, rank;
    uint32_t pad[4];
};
static_assert(sizeof(TRay) == 64, "64-byte ray");

struct TParams {
    const float *bricks;  // halo 1, x-y quads (4 floats per element, 16-byte aligned)
    int32_t N, B, nb;
    float sigmaMax;
    uint32_t seed;
    uint32_t spp;
    float *score;  // per global pixel: number of escaped paths
};

struct Cam {
    float eye[3], corner[3], du[3], dv[3];
};

__device__ __forceinline__ int32_t clampi(int32_t v, int32_t lo, int32_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int32_t owner_of(float px, float py, float pz, int32_t B, int32_t nb)
{
    const int32_t bx = clampi((int32_t)floorf(px / (float)B), 0, nb - 1);
    const int32_t by = clampi((int32_t)floorf(py / (float)B), 0, nb - 1);
    const int32_t bz = clampi((int32_t)floorf(pz / (float)B), 0, nb - 1);
    return bx + nb * (by + nb * bz);
}

// Trilinear sigma at p from the rank's brick of x-y quads (halo 1, origin
// org): the quad at (lo - org) along x and y holds both corners, clamped to
// the volume; the two z planes are clamped to the volume, then to the halo.
// Every evaluated point is owned by the rank, so the indices stay inside the
// halo, where this equals the unpartitioned trilinear sample.
__device__ __forceinline__ float sigma_at(const float4 *__restrict__ brick, int32_t N, int32_t S, const int32_t org[3],
                                          float px, float py, float pz)
{
    const float u[3] = {px - 0.5f, py - 0.5f, pz - 0.5f};
    int32_t j[3], z1 = 0;
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float fl = floorf(u[a]);
        f[a] = u[a] - fl;
        const int32_t lo = (int32_t)fl;
        if (a < 2) {
            j[a] = clampi(lo - org[a], 0, S - 1);
        } else {
            j[a] = clampi(clampi(lo, 0, N - 1) - org[a], 0, S - 1);
            z1 = clampi(clampi(lo + 1, 0, N - 1) - org[a], 0, S - 1);
        }
    }
    return quad_trilinear(brick, S, j[0], j[1], j[2], z1, f);
}

// Henyey-Greenstein (g = 0.3) scattering of direction d by (xi, xphi).
__device__ __forceinline__ void hg_scatter(float d[3], float xi, float xphi)
{
    const float g = 0.3f;
    const float s = (1.0f - g * g) / (1.0f - g + 2.0f * g * xi);
    float ct = (1.0f + g * g - s * s) / (2.0f * g);
    ct = fminf(1.0f, fmaxf(-1.0f, ct));
    const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
    const float phi = 6.2831853f * xphi;
    const float cp = cosf(phi), sp = sinf(phi);
    const float ax = fabsf(d[0]) < 0.9f ? 1.0f : 0.0f, ay = 1.0f - ax;
    float ux = d[1] * 0.0f - d[2] * ay, uy = d[2] * ax - d[0] * 0.0f, uz = d[0] * ay - d[1] * ax;
    const float ul = sqrtf(ux * ux + uy * uy + uz * uz);
    ux = ux / ul;
    uy = uy / ul;
    uz = uz / ul;
    const float vx = d[1] * uz - d[2] * uy, vy = d[2] * ux - d[0] * uz, vz = d[0] * uy - d[1] * ux;
    const float nx = (st * cp) * ux + (st * sp) * vx + ct * d[0];
    const float ny = (st * cp) * uy + (st * sp) * vy + ct * d[1];
    const float nz = (st * cp) * uz + (st * sp) * vz + ct * d[2];
    const float nl = sqrtf(nx * nx + ny * ny + nz * nz);
    d[0] = nx / nl;
    d[1] = ny / nl;
    d[2] = nz / nl;
}

// Advance path w on `rank` until it escapes, is absorbed, exceeds 64
// bounces, or must move to another rank.  Returns that rank, or -1 when it
// ended (an escape is scored).
__device__ int32_t track(const TParams &P, uint4 (&w)[4], int32_t rank)
{
    TRay r;
    *reinterpret_cast<uint4 *>(&r.px) = w[0];
    *reinterpret_cast<uint4 *>(&r.dy) = w[1];
    *reinterpret_cast<uint4 *>(&r.gpix) = w[2];
    *reinterpret_cast<uint4 *>(&r.pad[0]) = w[3];
    const int32_t S = P.B + 2;
    const int32_t bx = rank % P.nb, by = (rank / P.nb) % P.nb, bz = rank / (P.nb * P.nb);
    const int32_t org[3] = {bx * P.B - 1, by * P.B - 1, bz * P.B - 1};
    const float4 *brick = reinterpret_cast<const float4 *>(P.bricks) + (size_t)rank * S * S * S;
    const float fN = (float)P.N;
    float p[3] = {r.px, r.py, r.pz}, d[3] = {r.dx, r.dy, r.dz};
    int32_t dst = -1;
    for (;;) {
        const uint4 q4 = philox4x32_10(make_uint4(r.gpix, r.sample, r.bounce, r.event), make_uint2(P.seed, 7u));
        float q[3];
        if (r.pending) {
            q[0] = p[0];
            q[1] = p[1];
            q[2] = p[2];
            r.pending = 0u;
        } else {
            const float t = -logf(1.0f - u24(q4.x)) / P.sigmaMax;
            q[0] = p[0] + d[0] * t;
            q[1] = p[1] + d[1] * t;
            q[2] = p[2] + d[2] * t;
            if (!(q[0] >= 0.0f && q[0] < fN && q[1] >= 0.0f && q[1] < fN && q[2] >= 0.0f && q[2] < fN)) {
                atomicAdd(P.score + r.gpix, 1.0f);  // escaped: environment radiance 1
                break;
            }
            const int32_t own = owner_of(q[0], q[1], q[2], P.B, P.nb);
            if (own != rank) {
                p[0] = q[0];
                p[1] = q[1];
                p[2] = q[2];
                r.pending = 1u;
                dst = own;
                break;
            }
        }
        const float sg = sigma_at(brick, P.N, S, org, q[0], q[1], q[2]);
        p[0] = q[0];
        p[1] = q[1];
        p[2] = q[2];
        if (u24(q4.y) * P.sigmaMax < sg) {
            if (!(u24(q4.z) < 0.8f)) break;  // absorbed
            const uint4 h4 = philox4x32_10(make_uint4(r.gpix, r.sample, r.bounce, r.event), make_uint2(P.seed, 8u));
            r.bounce += 1u;
            if (r.bounce > 64u) break;
            hg_scatter(d, u24(q4.w), u24(h4.x));
            r.event = 0u;
        } else {
            r.event += 1u;
        }
    }
    r.px = p[0];
    r.py = p[1];
    r.pz = p[2];
    r.dx = d[0];
    r.dy = d[1];
    r.dz = d[2];
    r.rank = (uint32_t)dst;
    w[0] = *reinterpret_cast<const uint4 *>(&r.px);
    w[1] = *reinterpret_cast<const uint4 *>(&r.dy);
    w[2] = *reinterpret_cast<const uint4 *>(&r.gpix);
    w[3] = *reinterpret_cast<const uint4 *>(&r.pad[0]);
    return dst;
}

struct C4Work {
    static constexpr int V = 4;
    static constexpr bool kAppendRetired = false;
    static constexpr bool kDynamicWork = true;
    static constexpr bool kGridStride = false;
    static constexpr bool kFuseStep = false;
    static constexpr unsigned kStepReadMask = 0xfu;  // every vector
    static constexpr unsigned kStepWriteMask = 0xfu;
    static constexpr int kMinBlocksPerSM = 4;
    static constexpr int kItemsPerThread = 1;
    static constexpr int kBlock = kRoundsBlock;
    TParams P;
    __host__ __device__ uint32_t smemBytes() const { return 0u; }
    __device__ void load_smem(void *) const {}
    __device__ int32_t step(uint4 (&w)[4], int32_t rank, uint32_t, const void *) const { return track(P, w, rank); }
    __device__ void retire(const uint4 (&)[4]) const {}
};

// Shapes of the persistent kernel for this policy (the autotuner's
// candidates): {items per thread, CTAs per SM, threads}.  The work phase's
// occupancy is what matters here; the tile only sizes the scatter.
using C4Shapes = ShapeList<C4Work, Shape<C4Work, 1, 4, 256>, Shape<C4Work, 1, 3, 256>, Shape<C4Work, 1, 8, 128>,
                           Shape<C4Work, 2, 4, 256>>;


// Primary paths of one view: path (pixel, s) starts where its jittered ray
// enters the grid and is emitted, in out slot base + i, to that brick's rank
// (a ray that misses escapes at once).
__global__ void __launch_bounds__(kBlock) raygen_kernel(Cam cam, TParams P, int32_t W, int32_t H, uint32_t pixBase,
                                                        rf_device_queues q, unsigned long long slotBase)
{
    const uint32_t n = (uint32_t)W * H * P.spp;
    uint4 *outq = static_cast<uint4 *>(q.out);
    for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        const uint32_t pix = i / P.spp, s = i % P.spp;
        const int32_t x = (int32_t)(pix % (uint32_t)W), y = (int32_t)(pix / (uint32_t)W);
        const uint32_t gpix = pixBase + pix;
        const uint4 j = philox4x32_10(make_uint4(gpix, s, 0u, 0u), make_uint2(P.seed, 9u));
        const float px = (float)x + u24(j.x), py = (float)y + u24(j.y);
        float d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a] = cam.corner[a] + cam.du[a] * px + cam.dv[a] * py;
        const float len = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a] = d[a] / len;
        float tn[3], tf[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float ta = (0.0f - cam.eye[a]) / d[a];
            const float tb = ((float)P.N - cam.eye[a]) / d[a];
            tn[a] = fminf(ta, tb);
            tf[a] = fmaxf(ta, tb);
        }
        const float t0 = fmaxf(fmaxf(fmaxf(tn[0], tn[1]), tn[2]), 0.0f);
        const float t1 = fminf(fminf(tf[0], tf[1]), tf[2]);
        const unsigned long long slot = slotBase + i;
        if (!(t0 < t1)) {
            atomicAdd(P.score + gpix, 1.0f);
            q.dest[slot] = -1;
            continue;
        }
        TRay r;
        r.px = cam.eye[0] + d[0] * t0;
        r.py = cam.eye[1] + d[1] * t0;
        r.pz = cam.eye[2] + d[2] * t0;
        r.dx = d[0];
        r.dy = d[1];
        r.dz = d[2];
        r.bounce = 0u;
        r.event = 0u;
        r.gpix = gpix;
        r.sample = s;
        r.pending = 0u;
        r.rank = (uint32_t)owner_of(r.px, r.py, r.pz, P.B, P.nb);
        r.pad[0] = r.pad[1] = r.pad[2] = r.pad[3] = 0u;
        const uint4 *src = reinterpret_cast<const uint4 *>(&r);
#pragma unroll
        for (int k = 0; k < 4; ++k) outq[slot * 4 + k] = src[k];
        q.dest[slot] = (int32_t)r.rank;
    }
}

__global__ void set_count_kernel(unsigned long long *counter, unsigned long long n)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *counter = n;
}

// Plain per-rank kernel of one round: out slot i holds incoming path i when
// it moves on, destination -1 when it ended.
__global__ void __launch_bounds__(kBlock) track_kernel(TParams P, rf_device_queues q)
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
        uint4 w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = __ldg(inq + (size_t)i * 4 + k);
        const int32_t d = track(P, w, rf::rankOf(sOff, R, i));
        if (d >= 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) outq[(size_t)i * 4 + k] = w[k];
        }
        q.dest[i] = d;
    }
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
int c4_shapes(int32_t *out, int32_t cap)
{
    ShapeInfo v[C4Shapes::kCount];
    C4Shapes::infos(v);
    for (int i = 0; i < C4Shapes::kCount && i < cap; ++i) {
        out[3 * i] = v[i].block;
        out[3 * i + 1] = v[i].itemsPerThread;
        out[3 * i + 2] = v[i].ctasPerSM;
    }
    return C4Shapes::kCount;
}
}  // namespace rfi

extern "C" rf_status rf_c4_render(rf_ctx *ctx, const float *bricks, int32_t N, int32_t B, float sigmaMax,
                                  int32_t numViews, const float *cams, const int32_t *sizes, int32_t spp,
                                  uint32_t seed, float *score, int32_t batched, uint32_t maxRounds, void *stream,
                                  uint64_t *rounds, uint64_t *forwarded)
{
    if (!ctx || ctx->itemBytes != 64) {
        set_error("rf_c4_render: context of 64-byte paths required");
        return RF_ERR_ARG;
    }
    if (!bricks || !cams || !sizes || !score || numViews < 1 || spp < 1 || !(sigmaMax > 0.0f) || N < 1 || B < 1 ||
        N % B || (int64_t)(N / B) * (N / B) * (N / B) != ctx->numRanks || (reinterpret_cast<uintptr_t>(bricks) & 15u) ||
        batched < RF_FORM_HOST_LOOP || batched > RF_FORM_TUNED) {
        set_error("rf_c4_render: bad arguments");
        return RF_ERR_ARG;
    }
    uint64_t total = 0;
    for (int v = 0; v < numViews; ++v) total += (uint64_t)sizes[2 * v] * sizes[2 * v + 1] * spp;
    if (total > ctx->capacity || total > 0xFFFFFFFFull) {
        set_error("rf_c4_render: %llu paths exceed the capacity", (unsigned long long)total);
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TParams P;
    P.bricks = bricks;
    P.N = N;
    P.B = B;
    P.nb = N / B;
    P.sigmaMax = sigmaMax;
    P.seed = seed;
    P.spp = (uint32_t)spp;
    P.score = score;
    rf_device_queues q;
    rf_get_device_queues(ctx, &q);
    // every view's primary paths, in out slots by view, then one exchange
    unsigned long long slot = 0;
    uint32_t pixBase = 0;
    for (int v = 0; v < numViews; ++v) {
        Cam c;
        for (int a = 0; a < 3; ++a) {
            c.eye[a] = cams[12 * v + a];
            c.corner[a] = cams[12 * v + 3 + a];
            c.du[a] = cams[12 * v + 6 + a];
            c.dv[a] = cams[12 * v + 9 + a];
        }
        const int32_t W = sizes[2 * v], H = sizes[2 * v + 1];
        const uint64_t n = (uint64_t)W * H * spp;
        raygen_kernel<<<grid_for(ctx, n), kBlock, 0, s>>>(c, P, W, H, pixBase, q, slot);
        RF_LAUNCHED("c4 raygen_kernel");
        slot += n;
        pixBase += (uint32_t)(W * H);
    }
    set_count_kernel<<<1, 32, 0, s>>>(q.outCount, total);
    RF_LAUNCHED("c4 set_count_kernel");
    // RF_FORM_TUNED: the form the context holds for this policy (set by the autotuner)
    const int32_t form = batched == RF_FORM_TUNED ? ctx->batchedForm[RF_POLICY_TRANSPORT] : batched;
    uint64_t active = 0, fwd = 0, r = 0;
    if (form == RF_FORM_GRAPH) {
        // graph form: the tracking kernel and the exchange repeated by a while node
        if (rf_status st = rf_exchange(ctx, stream, nullptr)) return st;
        rf_status st = run_graph_loop(ctx, s, maxRounds, [&](cudaStream_t cs) -> rf_status {
            track_kernel<<<grid_for(ctx, ctx->capacity), kBlock, 0, cs>>>(P, q);
            RF_LAUNCHED("c4 track_kernel");
            return launch_exchange(ctx, cs);
        }, &r, &fwd);
        if (st != RF_OK) return st;
        active = ctx->host->numActive;
    } else if (form == RF_FORM_PERSISTENT) {
        if (rf_status st = rf_exchange(ctx, stream, nullptr)) return st;
        C4Work w;
        w.P = P;
        unsigned long long res[4];
        rf_status st = C4Shapes::launch(ctx->batchedShape[RF_POLICY_TRANSPORT], ctx, w, maxRounds, s, nullptr, 0u,
                                        nullptr, 0ull, nullptr, res);
        if (st != RF_OK) return st;
        r = res[0];
        fwd = res[1];
        active = ctx->host->numActive;
    } else {
        rf_status st = rf_exchange(ctx, stream, &active);
        if (st != RF_OK) return st;
        while (active > 0 && r < maxRounds) {
            time_begin(ctx, kTimeWork, s);
            track_kernel<<<grid_for(ctx, ctx->capacity), kBlock, 0, s>>>(P, q);
            RF_LAUNCHED("c4 track_kernel");
            time_end(ctx, kTimeWork, s);
            if ((st = rf_exchange(ctx, stream, &active))) return st;
            fwd += active;
            ++r;
        }
    }
    if (rounds) *rounds = r;
    if (forwarded) *forwarded = fwd;
    if (active) {
        set_error("rf_c4_render: %llu paths still active after %u rounds", (unsigned long long)active, maxRounds);
        return RF_ERR_MAX_ROUNDS;
    }
    return RF_OK;
}
