// Absorption marching through a brick-partitioned density grid: the VoPaT
// style data-parallel trace (Sec. 5.1, Fig. 1) with the RaFI interface.
// Every logical rank owns one brick of an N^3 float grid (plus a one-voxel
// halo, so trilinear taps near a face stay local).  Raygen forwards each
// primary ray to the brick of its first sample; the trace kernel marches a
// ray through its rank's brick at step 0.5 and forwards it to the next brick
// when a sample leaves its own, or writes T = expf(-tau) when it leaves the
// volume.  Forwarding does not change what is computed (Sec. 5.1): tau is the
// same sum, in the same order, as marching the unpartitioned grid.
//
// Built with -fmad=false: positions, owners and tau follow the written
// operation order exactly.
#include <cstring>

#include "internal.cuh"
#include "rafi_device.cuh"

namespace rfi {
namespace {

constexpr int kBlock = 256;

// 48-byte ray: origin, direction, next sample index k, tau so far, pixel,
// current rank, and the entry/exit distances of the volume box.
struct __align__(16) Ray {
    float ox, oy, oz;
    float dx, dy, dz;
    float k;
    float tau;
    int32_t pixel;
    int32_t rank;
    float t0, t1;
};
static_assert(sizeof(Ray) == 48, "48-byte ray");

struct Cam {
    float eye[3], corner[3], du[3], dv[3];
};

__device__ __forceinline__ int32_t clampi(int32_t v, int32_t lo, int32_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int32_t brick_of(float p, int32_t B, int32_t nb)
{
    return clampi((int32_t)floorf(p / (float)B), 0, nb - 1);
}

__device__ __forceinline__ int32_t owner(float px, float py, float pz, int32_t B, int32_t nb)
{
    return brick_of(px, B, nb) + nb * (brick_of(py, B, nb) + nb * brick_of(pz, B, nb));
}

// Trilinear sigma at p from the brick (bx,by,bz) stored with halo as x-y
// quads: voxel centres at v + 0.5, clamp to the volume edge.  The quad at
// (lo - origin) along x and y carries both corners, clamped to the volume;
// along z the two planes are clamped to the volume, then to the halo.  A
// sample the rank owns lies within its brick, so the indices stay inside
// the halo, where this equals the unpartitioned trilinear sample.
__device__ __forceinline__ float sample(const float4 *__restrict__ brick, int32_t N, int32_t B, int32_t bx,
                                        int32_t by, int32_t bz, float px, float py, float pz)
{
    const int32_t S = B + 2;
    const float u[3] = {px - 0.5f, py - 0.5f, pz - 0.5f};
    const int32_t org[3] = {bx * B - 1, by * B - 1, bz * B - 1};
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

// Element (lx, ly, lz) of brick r: the x-y quad of the volume voxels at the
// brick's halo origin + (lx, ly, lz), each index clamped to the volume.
__global__ void __launch_bounds__(kBlock) make_bricks_kernel(const float *__restrict__ vol, int32_t N, int32_t B,
                                                             float4 *__restrict__ bricks)
{
    const int32_t nb = N / B, S = B + 2;
    const uint64_t per = (uint64_t)S * S * S;
    const uint64_t total = per * nb * nb * nb;
    for (uint64_t v = blockIdx.x * (uint64_t)kBlock + threadIdx.x; v < total; v += (uint64_t)gridDim.x * kBlock) {
        const int32_t r = (int32_t)(v / per);
        const int32_t l = (int32_t)(v % per);
        const int32_t lx = l % S, ly = (l / S) % S, lz = l / (S * S);
        const int32_t bx = r % nb, by = (r / nb) % nb, bz = r / (nb * nb);
        const int32_t gx = clampi(bx * B - 1 + lx, 0, N - 1), gx1 = clampi(bx * B + lx, 0, N - 1);
        const int32_t gy = clampi(by * B - 1 + ly, 0, N - 1), gy1 = clampi(by * B + ly, 0, N - 1);
        const int32_t gz = clampi(bz * B - 1 + lz, 0, N - 1);
        const float *pl = vol + (size_t)gz * N * N;
        bricks[v] = make_float4(pl[(size_t)gy * N + gx], pl[(size_t)gy * N + gx1], pl[(size_t)gy1 * N + gx],
                                pl[(size_t)gy1 * N + gx1]);
    }
}

__global__ void __launch_bounds__(kBlock) raygen_kernel(Cam cam, int32_t N, int32_t B, int32_t W, int32_t H,
                                                        float *image, int32_t *hopCount, rf_device_queues q)
{
    const int32_t pix = blockIdx.x * kBlock + threadIdx.x;
    if (pix >= W * H) return;
    if (hopCount) hopCount[pix] = 0;
    const int32_t x = pix % W, y = pix / W;
    const float px = (float)x + 0.5f, py = (float)y + 0.5f;
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
        const float tb = ((float)N - cam.eye[a]) / d[a];
        tn[a] = fminf(ta, tb);
        tf[a] = fmaxf(ta, tb);
    }
    const float t0 = fmaxf(fmaxf(fmaxf(tn[0], tn[1]), tn[2]), 0.0f);
    const float t1 = fminf(fminf(tf[0], tf[1]), tf[2]);
    const float tk = t0 + (0.0f + 0.5f) * 0.5f;
    if (!(tk < t1)) {
        image[pix] = 1.0f;
        return;
    }
    const int32_t nb = N / B;
    Ray r;
    r.ox = cam.eye[0];
    r.oy = cam.eye[1];
    r.oz = cam.eye[2];
    r.dx = d[0];
    r.dy = d[1];
    r.dz = d[2];
    r.k = 0.0f;
    r.tau = 0.0f;
    r.pixel = pix;
    r.t0 = t0;
    r.t1 = t1;
    r.rank = owner(r.ox + r.dx * tk, r.oy + r.dy * tk, r.oz + r.dz * tk, B, nb);
    rf::forward(q, r, r.rank);
}

__global__ void __launch_bounds__(kBlock) march_kernel(const float *__restrict__ bricks, int32_t N, int32_t B,
                                                       float *image, int32_t *hopLog, int32_t maxHops,
                                                       int32_t *hopCount, rf_device_queues q)
{
    __shared__ uint32_t sOff[RF_MAX_RANKS + 1];
    const int32_t R = q.numRanks;
    for (int e = threadIdx.x; e <= R; e += kBlock) sOff[e] = q.inOffset[e];
    __syncthreads();
    const uint32_t n = sOff[R];
    const int32_t nb = N / B, S = B + 2;
    for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        const int32_t rank = rf::rankOf(sOff, R, i);
        Ray r = rf::getIncoming<Ray>(q, i);
        if (hopCount) {
            const int32_t c = hopCount[r.pixel];
            if (hopLog && c < maxHops) hopLog[(size_t)r.pixel * maxHops + c] = rank;
            hopCount[r.pixel] = c + 1;
        }
        const int32_t bx = rank % nb, by = (rank / nb) % nb, bz = rank / (nb * nb);
        const float4 *brick = reinterpret_cast<const float4 *>(bricks) + (size_t)rank * S * S * S;
        int32_t k = (int32_t)r.k;
        float tau = r.tau;
        for (;;) {
            const float tk = r.t0 + ((float)k + 0.5f) * 0.5f;
            if (!(tk < r.t1)) {
                image[r.pixel] = expf(-tau);
                break;
            }
            const float px = r.ox + r.dx * tk, py = r.oy + r.dy * tk, pz = r.oz + r.dz * tk;
            const int32_t own = owner(px, py, pz, B, nb);
            if (own != rank) {
                r.k = (float)k;
                r.tau = tau;
                r.rank = own;
                rf::forward(q, r, own);
                break;
            }
            tau = tau + sample(brick, N, B, bx, by, bz, px, py, pz) * 0.5f;
            ++k;
        }
    }
}

rf_status check_c0(rf_ctx *ctx, int32_t N, int32_t B, const char *fn)
{
    if (!ctx) {
        set_error("%s: NULL context", fn);
        return RF_ERR_ARG;
    }
    if (ctx->itemBytes != sizeof(Ray)) {
        set_error("%s: rays are %zu bytes (context has %u)", fn, sizeof(Ray), ctx->itemBytes);
        return RF_ERR_ARG;
    }
    if (N < 1 || B < 1 || N % B || (int64_t)(N / B) * (N / B) * (N / B) != ctx->numRanks) {
        set_error("%s: N %d, brick %d do not give %d ranks", fn, N, B, ctx->numRanks);
        return RF_ERR_ARG;
    }
    return RF_OK;
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

extern "C" {

rf_status rf_c0_make_bricks(const float *volume, int32_t N, int32_t B, float *bricks, void *stream)
{
    if (!volume || !bricks || N < 1 || B < 1 || N % B || (reinterpret_cast<uintptr_t>(bricks) & 15u)) {
        set_error("rf_c0_make_bricks: bad arguments (bricks must be 16-byte aligned)");
        return RF_ERR_ARG;
    }
    const int32_t nb = N / B, S = B + 2;
    const uint64_t total = (uint64_t)S * S * S * nb * nb * nb;
    uint64_t blocks = (total + kBlock - 1) / kBlock;
    if (blocks > 65535u * 16u) blocks = 65535u * 16u;
    make_bricks_kernel<<<(unsigned)blocks, kBlock, 0, static_cast<cudaStream_t>(stream)>>>(
        volume, N, B, reinterpret_cast<float4 *>(bricks));
    RF_LAUNCHED("make_bricks_kernel");
    return RF_OK;
}

rf_status rf_c0_raygen(rf_ctx *ctx, const float *cam, int32_t N, int32_t B, int32_t W, int32_t H, float *image,
                       void *stream)
{
    if (rf_status st = check_c0(ctx, N, B, "rf_c0_raygen")) return st;
    if (!cam || !image || W < 1 || H < 1 || (uint64_t)W * H > ctx->capacity) {
        set_error("rf_c0_raygen: bad camera/image or W*H above capacity");
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    Cam c;
    for (int a = 0; a < 3; ++a) {
        c.eye[a] = cam[a];
        c.corner[a] = cam[3 + a];
        c.du[a] = cam[6 + a];
        c.dv[a] = cam[9 + a];
    }
    rf_device_queues q;
    rf_get_device_queues(ctx, &q);
    const int blocks = (W * H + kBlock - 1) / kBlock;
    raygen_kernel<<<blocks, kBlock, 0, static_cast<cudaStream_t>(stream)>>>(c, N, B, W, H, image, nullptr, q);
    RF_LAUNCHED("raygen_kernel");
    return RF_OK;
}

rf_status rf_c0_march(rf_ctx *ctx, const float *bricks, int32_t N, int32_t B, float *image, int32_t *hopLog,
                      int32_t maxHops, int32_t *hopCount, void *stream)
{
    if (rf_status st = check_c0(ctx, N, B, "rf_c0_march")) return st;
    if (!bricks || !image || (hopLog && (!hopCount || maxHops < 1)) || (reinterpret_cast<uintptr_t>(bricks) & 15u)) {
        set_error("rf_c0_march: NULL or unaligned bricks, NULL image, or hopLog without hopCount");
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    rf_device_queues q;
    rf_get_device_queues(ctx, &q);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    time_begin(ctx, kTimeWork, s);
    march_kernel<<<grid_for(ctx, ctx->capacity), kBlock, 0, s>>>(bricks, N, B, image, hopLog, maxHops, hopCount, q);
    RF_LAUNCHED("march_kernel");
    time_end(ctx, kTimeWork, s);
    return RF_OK;
}

rf_status rf_c0_render(rf_ctx *ctx, const float *bricks, const float *cam, int32_t N, int32_t B, int32_t W,
                       int32_t H, float *image, int32_t *hopLog, int32_t maxHops, int32_t *hopCount,
                       uint32_t maxRounds, void *stream, uint64_t *rounds)
{
    if (rf_status st = check_c0(ctx, N, B, "rf_c0_render")) return st;
    if (!cam || !image || !bricks || W < 1 || H < 1 || (uint64_t)W * H > ctx->capacity ||
        (hopLog && (!hopCount || maxHops < 1))) {
        set_error("rf_c0_render: bad arguments");
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    Cam c;
    for (int a = 0; a < 3; ++a) {
        c.eye[a] = cam[a];
        c.corner[a] = cam[3 + a];
        c.du[a] = cam[6 + a];
        c.dv[a] = cam[9 + a];
    }
    rf_device_queues q;
    rf_get_device_queues(ctx, &q);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = (W * H + kBlock - 1) / kBlock;
    raygen_kernel<<<blocks, kBlock, 0, s>>>(c, N, B, W, H, image, hopCount, q);
    RF_LAUNCHED("raygen_kernel");
    uint64_t active = 0, r = 0;
    rf_status st = rf_exchange(ctx, stream, &active);
    if (st != RF_OK) return st;
    while (active > 0) {
        if (r >= maxRounds) {
            set_error("rf_c0_render: %llu rays still active after %u rounds", (unsigned long long)active, maxRounds);
            if (rounds) *rounds = r;
            return RF_ERR_MAX_ROUNDS;
        }
        st = rf_c0_march(ctx, bricks, N, B, image, hopLog, maxHops, hopCount, stream);
        if (st != RF_OK) return st;
        st = rf_exchange(ctx, stream, &active);
        if (st != RF_OK) return st;
        ++r;
    }
    if (rounds) *rounds = r;
    return RF_OK;
}

rf_status rf_c0_render_graph(rf_ctx *ctx, const float *bricks, const float *cam, int32_t N, int32_t B, int32_t W,
                             int32_t H, float *image, int32_t *hopLog, int32_t maxHops, int32_t *hopCount,
                             uint32_t maxRounds, void *stream, uint64_t *rounds)
{
    if (rf_status st = check_c0(ctx, N, B, "rf_c0_render_graph")) return st;
    if (!cam || !image || !bricks || W < 1 || H < 1 || (uint64_t)W * H > ctx->capacity ||
        (hopLog && (!hopCount || maxHops < 1))) {
        set_error("rf_c0_render_graph: bad arguments");
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    Cam c;
    for (int a = 0; a < 3; ++a) {
        c.eye[a] = cam[a];
        c.corner[a] = cam[3 + a];
        c.du[a] = cam[6 + a];
        c.dv[a] = cam[9 + a];
    }
    rf_device_queues q;
    rf_get_device_queues(ctx, &q);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = (W * H + kBlock - 1) / kBlock;
    // every pointer and value the captured kernels take
    struct Key {
        const float *bricks;
        float cam[12];
        int32_t N, B, W, H, maxHops;
        float *image;
        int32_t *hopLog, *hopCount;
    } key;
    memset(&key, 0, sizeof key);
    key.bricks = bricks;
    for (int a = 0; a < 12; ++a) key.cam[a] = cam[a];
    key.N = N;
    key.B = B;
    key.W = W;
    key.H = H;
    key.maxHops = maxHops;
    key.image = image;
    key.hopLog = hopLog;
    key.hopCount = hopCount;
    uint64_t r = 0;
    rf_status st = run_graph_loop(
        ctx, s, maxRounds,
        [&](cudaStream_t cs) -> rf_status {
            if (rf_status ms = rf_c0_march(ctx, bricks, N, B, image, hopLog, maxHops, hopCount, cs)) return ms;
            return launch_exchange(ctx, cs);
        },
        &r, nullptr,
        [&](cudaStream_t cs) -> rf_status {
            raygen_kernel<<<blocks, kBlock, 0, cs>>>(c, N, B, W, H, image, hopCount, q);
            RF_LAUNCHED("raygen_kernel");
            return launch_exchange(ctx, cs);
        },
        &key, sizeof key);
    if (st != RF_OK) return st;
    if (rounds) *rounds = r;
    if (ctx->host->numActive) {
        set_error("rf_c0_render_graph: %llu rays still active after %u rounds",
                  (unsigned long long)ctx->host->numActive, maxRounds);
        return RF_ERR_MAX_ROUNDS;
    }
    return RF_OK;
}

}  // extern "C"
