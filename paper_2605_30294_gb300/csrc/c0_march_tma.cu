// Absorption marching with each rank's brick staged whole in shared memory
// by the tensor memory accelerator (cp.async.bulk.tensor), the alternative to
// c0_march.cu's quad bricks read through L1.  Same rays, same samples, same
// corners and the same float operations in the same order: the image is
// bit-identical to rf_c0_render's.
//
// Each CTA takes a chunk of one rank's incoming segment, loads that rank's
// brick (a scalar copy with a one-voxel halo, rows padded to a multiple of
// 16 bytes as TMA wants) into shared memory with one 3-D tensor copy, and
// marches its rays from there; rays that leave the brick are forwarded as in
// c0_march.cu.  A 32^3 brick with halo is 36 x 34 x 34 floats (166 KB), so
// one CTA fills an SM's shared memory.
//
// Built with -fmad=false, like c0_march.cu.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "internal.cuh"
#include "rafi_device.cuh"

namespace rfi {
namespace {

constexpr int kBlock = 256;
constexpr uint32_t kChunk = 256;  // rays per CTA

struct __align__(16) Ray {  // the 48-byte ray of c0_march.cu
    float ox, oy, oz;
    float dx, dy, dz;
    float k;
    float tau;
    int32_t pixel;
    int32_t rank;
    float t0, t1;
};
static_assert(sizeof(Ray) == 48, "48-byte ray");

__device__ __forceinline__ int32_t clampi(int32_t v, int32_t lo, int32_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

__host__ __device__ inline int32_t row_floats(int32_t B) { return (B + 2 + 3) / 4 * 4; }

__device__ __forceinline__ int32_t owner(float px, float py, float pz, int32_t B, int32_t nb)
{
    const int32_t bx = clampi((int32_t)floorf(px / (float)B), 0, nb - 1);
    const int32_t by = clampi((int32_t)floorf(py / (float)B), 0, nb - 1);
    const int32_t bz = clampi((int32_t)floorf(pz / (float)B), 0, nb - 1);
    return bx + nb * (by + nb * bz);
}

// Scalar brick r: element (lx, ly, lz), lx < row_floats(B), holds the voxel at
// the brick's halo origin + (lx, ly, lz), each index clamped to the volume.
__global__ void __launch_bounds__(kBlock) make_scalar_bricks_kernel(const float *__restrict__ vol, int32_t N,
                                                                    int32_t B, float *__restrict__ bricks)
{
    const int32_t nb = N / B, S = B + 2, X = row_floats(B);
    const uint64_t per = (uint64_t)X * S * S;
    const uint64_t total = per * nb * nb * nb;
    for (uint64_t v = blockIdx.x * (uint64_t)kBlock + threadIdx.x; v < total; v += (uint64_t)gridDim.x * kBlock) {
        const int32_t r = (int32_t)(v / per);
        const int32_t l = (int32_t)(v % per);
        const int32_t lx = l % X, ly = (l / X) % S, lz = l / (X * S);
        const int32_t bx = r % nb, by = (r / nb) % nb, bz = r / (nb * nb);
        const int32_t gx = clampi(bx * B - 1 + lx, 0, N - 1);
        const int32_t gy = clampi(by * B - 1 + ly, 0, N - 1);
        const int32_t gz = clampi(bz * B - 1 + lz, 0, N - 1);
        bricks[v] = vol[((size_t)gz * N + gy) * N + gx];
    }
}

// Trilinear sigma from the staged scalar brick s (X floats per row, S rows
// per plane), with the corners and the blend order of quad_trilinear: x, then
// y, then z.
__device__ __forceinline__ float sample_smem(const float *s, int32_t X, int32_t S, int32_t N, const int32_t org[3],
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
    const float *p0 = s + ((size_t)j[2] * S + j[1]) * X + j[0];
    const float *p1 = s + ((size_t)z1 * S + j[1]) * X + j[0];
    const float gx = 1.0f - f[0], gy = 1.0f - f[1], gz = 1.0f - f[2];
    const float c00 = p0[0] * gx + p0[1] * f[0];
    const float c10 = p0[X] * gx + p0[X + 1] * f[0];
    const float c01 = p1[0] * gx + p1[1] * f[0];
    const float c11 = p1[X] * gx + p1[X + 1] * f[0];
    const float c0 = c00 * gy + c10 * f[1];
    const float c1 = c01 * gy + c11 * f[1];
    return c0 * gz + c1 * f[2];
}

__global__ void __launch_bounds__(kBlock, 1) march_tma_kernel(const __grid_constant__ CUtensorMap tmap, int32_t N,
                                                              int32_t B, float *image, rf_device_queues q,
                                                              unsigned int *status)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ int32_t sRank;
    __shared__ uint32_t sLo, sHi;
    const int32_t R = q.numRanks, nb = N / B, S = B + 2, X = row_floats(B);
    if (threadIdx.x == 0) {
        // this CTA's (rank, chunk): chunks of kChunk rays, rank after rank
        uint32_t b = blockIdx.x;
        sRank = -1;
        for (int32_t r = 0; r < R; ++r) {
            const uint32_t lo = q.inOffset[r], hi = q.inOffset[r + 1];
            const uint32_t nch = (hi - lo + kChunk - 1) / kChunk;
            if (b < nch) {
                sRank = r;
                sLo = lo + b * kChunk;
                sHi = min(hi, sLo + kChunk);
                break;
            }
            b -= nch;
        }
        if (sRank >= 0) {
            mbar_init(&bar, 1);
            fence_proxy_async_smem();
            const uint32_t bytes = (uint32_t)X * S * S * 4u;
            mbar_arrive_expect_tx(&bar, bytes);
            const int32_t zc = sRank * S;
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4}], [%5];" ::"r"(smem_u32(smem)),
                "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(0), "r"(0), "r"(zc), "r"(smem_u32(&bar))
                : "memory");
        }
    }
    __syncthreads();
    const int32_t rank = sRank;
    if (rank < 0) return;
    const bool ok = mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(!ok)) {
        // give the copy one more bounded wait to land before the CTA leaves
        if (threadIdx.x == 0) {
            atomicOr(status, RF_DEV_TIMEOUT);
            (void)mbar_wait_bounded(&bar, 0);
        }
        __syncthreads();
        return;
    }
    const float *s = reinterpret_cast<const float *>(smem);
    const int32_t bx = rank % nb, by = (rank / nb) % nb, bz = rank / (nb * nb);
    const int32_t org[3] = {bx * B - 1, by * B - 1, bz * B - 1};
    for (uint32_t i = sLo + threadIdx.x; i < sHi; i += kBlock) {
        Ray r = rf::getIncoming<Ray>(q, i);
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
            tau = tau + sample_smem(s, X, S, N, org, px, py, pz) * 0.5f;
            ++k;
        }
    }
}

// The driver's tensor-map encoder, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            (void)cudaGetLastError();
    });
    return fn;
}

// Everything a march launch takes, checked and encoded outside any stream capture.
struct TmaMarch {
    CUtensorMap tmap;
    const float *bricks;
    int32_t N, B;
    float *image;
    size_t smem;
    unsigned chunks;
};

rf_status prepare_tma(rf_ctx *ctx, const float *scalarBricks, int32_t N, int32_t B, float *image, const char *fn,
                      TmaMarch &m)
{
    if (!ctx || ctx->itemBytes != sizeof(Ray)) {
        set_error("%s: context of 48-byte rays required", fn);
        return RF_ERR_ARG;
    }
    if (!scalarBricks || !image || N < 1 || B < 1 || N % B || (int64_t)(N / B) * (N / B) * (N / B) != ctx->numRanks ||
        (reinterpret_cast<uintptr_t>(scalarBricks) & 15u) || B + 2 > 256) {
        set_error("%s: bad arguments (bricks 16-byte aligned, B + 2 <= 256)", fn);
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    const int32_t S = B + 2, X = row_floats(B), R = ctx->numRanks;
    m.smem = (size_t)X * S * S * 4u;
    int optin = 0;
    RF_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    if (m.smem + 64 > (size_t)optin) {
        set_error("%s: a %d^3 brick with halo (%zu bytes) does not fit in shared memory (%d)", fn, B, m.smem, optin);
        return RF_ERR_ARG;
    }
    auto enc = encoder();
    if (!enc) {
        set_error("%s: cuTensorMapEncodeTiled is not available", fn);
        return RF_ERR_CUDA;
    }
    // the bricks as one 3-D tensor: x (padded rows), y, and z of all bricks in turn
    const cuuint64_t dims[3] = {(cuuint64_t)X, (cuuint64_t)S, (cuuint64_t)S * R};
    const cuuint64_t strides[2] = {(cuuint64_t)X * 4u, (cuuint64_t)X * S * 4u};
    const cuuint32_t box[3] = {(cuuint32_t)X, (cuuint32_t)S, (cuuint32_t)S};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult cr = enc(&m.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(scalarBricks), dims,
                            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        set_error("%s: cuTensorMapEncodeTiled failed (%d)", fn, (int)cr);
        return RF_ERR_CUDA;
    }
    RF_CUDA(cudaFuncSetAttribute(march_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m.smem));
    m.bricks = scalarBricks;
    m.N = N;
    m.B = B;
    m.image = image;
    // an upper bound on the chunks of all ranks' segments
    m.chunks = (unsigned)((ctx->capacity + kChunk - 1) / kChunk + (uint64_t)R);
    return RF_OK;
}

rf_status launch_tma(rf_ctx *ctx, const TmaMarch &m, cudaStream_t s)
{
    rf_device_queues q;
    rf_get_device_queues(ctx, &q);
    time_begin(ctx, kTimeWork, s);
    march_tma_kernel<<<m.chunks, kBlock, m.smem, s>>>(m.tmap, m.N, m.B, m.image, q, &ctx->dev->status);
    RF_LAUNCHED("march_tma_kernel");
    time_end(ctx, kTimeWork, s);
    return RF_OK;
}

}  // namespace
}  // namespace rfi

using namespace rfi;

extern "C" {

rf_status rf_c0_make_scalar_bricks(const float *volume, int32_t N, int32_t B, float *bricks, void *stream)
{
    if (!volume || !bricks || N < 1 || B < 1 || N % B || (reinterpret_cast<uintptr_t>(bricks) & 15u)) {
        set_error("rf_c0_make_scalar_bricks: bad arguments (bricks must be 16-byte aligned)");
        return RF_ERR_ARG;
    }
    const int32_t nb = N / B, S = B + 2;
    const uint64_t total = (uint64_t)row_floats(B) * S * S * nb * nb * nb;
    uint64_t blocks = (total + kBlock - 1) / kBlock;
    if (blocks > 65535u * 16u) blocks = 65535u * 16u;
    make_scalar_bricks_kernel<<<(unsigned)blocks, kBlock, 0, static_cast<cudaStream_t>(stream)>>>(volume, N, B,
                                                                                                     bricks);
    RF_LAUNCHED("make_scalar_bricks_kernel");
    return RF_OK;
}

rf_status rf_c0_march_tma(rf_ctx *ctx, const float *scalarBricks, int32_t N, int32_t B, float *image, void *stream)
{
    TmaMarch m;
    if (rf_status st = prepare_tma(ctx, scalarBricks, N, B, image, "rf_c0_march_tma", m)) return st;
    DeviceGuard g(ctx->device);
    return launch_tma(ctx, m, static_cast<cudaStream_t>(stream));
}

rf_status rf_c0_render_tma(rf_ctx *ctx, const float *scalarBricks, const float *cam, int32_t N, int32_t B, int32_t W,
                           int32_t H, float *image, int32_t form, uint32_t maxRounds, void *stream, uint64_t *rounds)
{
    if (form != RF_FORM_HOST_LOOP && form != RF_FORM_GRAPH) {
        set_error("rf_c0_render_tma: form %d is neither the host loop nor the graph loop", form);
        return RF_ERR_ARG;
    }
    TmaMarch m;
    if (rf_status st = prepare_tma(ctx, scalarBricks, N, B, image, "rf_c0_render_tma", m)) return st;
    if (!cam || W < 1 || H < 1 || (uint64_t)W * H > ctx->capacity) {
        set_error("rf_c0_render_tma: bad camera or W*H above capacity");
        return RF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t r = 0;
    if (form == RF_FORM_GRAPH) {
        // the march and the exchange repeated by a conditional while node; raygen
        // and the first exchange run in the graph before the loop
        struct Key {
            const float *bricks;
            float cam[12];
            int32_t N, B, W, H;
            float *image;
        } key;
        memset(&key, 0, sizeof key);
        key.bricks = scalarBricks;
        for (int a = 0; a < 12; ++a) key.cam[a] = cam[a];
        key.N = N;
        key.B = B;
        key.W = W;
        key.H = H;
        key.image = image;
        rf_status st = run_graph_loop(
            ctx, s, maxRounds,
            [&](cudaStream_t cs) -> rf_status {
                if (rf_status ms = launch_tma(ctx, m, cs)) return ms;
                return launch_exchange(ctx, cs);
            },
            &r, nullptr,
            [&](cudaStream_t cs) -> rf_status {
                if (rf_status rs = rf_c0_raygen(ctx, cam, N, B, W, H, image, cs)) return rs;
                return launch_exchange(ctx, cs);
            },
            &key, sizeof key);
        if (st != RF_OK) return st;
        if (rounds) *rounds = r;
        if (ctx->host->numActive) {
            set_error("rf_c0_render_tma: %llu rays still active after %u rounds",
                      (unsigned long long)ctx->host->numActive, maxRounds);
            return RF_ERR_MAX_ROUNDS;
        }
        return RF_OK;
    }
    if (rf_status st = rf_c0_raygen(ctx, cam, N, B, W, H, image, stream)) return st;
    uint64_t active = 0;
    rf_status st = rf_exchange(ctx, stream, &active);
    if (st != RF_OK) return st;
    while (active > 0) {
        if (r >= maxRounds) {
            set_error("rf_c0_render_tma: %llu rays still active after %u rounds", (unsigned long long)active,
                      maxRounds);
            if (rounds) *rounds = r;
            return RF_ERR_MAX_ROUNDS;
        }
        if ((st = launch_tma(ctx, m, s))) return st;
        if ((st = rf_exchange(ctx, stream, &active))) return st;
        ++r;
    }
    if (rounds) *rounds = r;
    return RF_OK;
}

}  // extern "C"
