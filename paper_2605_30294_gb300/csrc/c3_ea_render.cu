// Differentiable emission-absorption rendering through a brick-partitioned
// density grid: the Lander renderer's integration model (Sec. 5.2, each ray
// carries its accumulated colour and transmittance across partitions) with a
// hand-written adjoint.
//
// Forward: spp jittered rays per pixel; per sample sigma_k (trilinear),
// e_k = expf(-sigma_k/2), alpha_k = 1 - e_k, c_k = 20 sigma_k,
// C += (T alpha_k) c_k, T *= e_k; rays are forwarded to the next brick.
//
// Adjoint: dC/dsigma_k = T_k (0.5 e_k c_k + 20 alpha_k) - 0.5 S_{>k} with
// S_{>k} = sum_{j>k} T_j alpha_j c_j = C - sum_{j<=k} T_j alpha_j c_j.  An
// adjoint ray carries the final C of its forward ray and dL/dC; walking the
// same bricks it recomputes T_k and the running suffix segment by segment (no
// stored history, no division by 1 - alpha) and scatters dL/dC * dC/dsigma_k
// with the trilinear weights into the gradient grid (atomic adds, summed per
// ray over consecutive samples that share their eight corners).
//
// Late samples of an opaque ray have a suffix far below C, so C minus a float
// prefix loses most of its digits.  Both passes therefore keep their sums as
// unevaluated pairs (hi + lo, Knuth's error-free TwoSum): the forward adds
// each T alpha c to (C, Clo) and may return Clo beside C (C itself is the
// plain float sum, bit for bit); the adjoint starts from (C, Clo) and takes
// each T alpha c off again, so the suffix it uses is exact up to the rounding
// of the individual terms.  The derivative's alpha term takes alpha from
// expm1f (1 - e loses it where sigma is tiny); the suffix keeps subtracting
// the forward's own float terms.
//
// Built with -fmad=false (the written float order, as the oracle's).
#include "internal.cuh"
#include "philox.cuh"
#include "rafi_device.cuh"

namespace rfi {
namespace {

constexpr int kBlock = 256;

// 64-byte ray.  Forward: (acc, lo) = C so far as a hi + lo pair.  Adjoint:
// (acc, lo) = the suffix still to come (C minus the terms walked so far),
// cfin = C of the forward ray, g = dL/dC.
struct __align__(16) EARay {
    float ox, oy, oz, dx;
    float dy, dz, k, T;
    float acc, t0, t1;
    uint32_t id;
    float cfin, g;
    int32_t rank;
    uint32_t lo;  // float bits of the low part of acc
};
static_assert(sizeof(EARay) == 64, "64-byte ray");

struct Cam {
    float eye[3], corner[3], du[3], dv[3];
};

struct EAParams {
    const float *bricks;
    int32_t N, B, nb;
    int32_t W, H, spp;
    uint32_t seed;
    float *rayC;        // W*H*spp
    float *rayCLo;      // W*H*spp low parts of rayC (nullable)
    float *grad;        // N^3 (adjoint)
    const float *gimg;  // W*H dL/dpixel (adjoint)
};

// a + b = s + err exactly (Knuth's TwoSum; the file is built without FMA
// contraction, so every operation rounds once)
__device__ __forceinline__ float two_sum(float a, float b, float &err)
{
    const float s = a + b;
    const float bp = s - a;
    const float ap = s - bp;
    err = (a - ap) + (b - bp);
    return s;
}

__device__ __forceinline__ int32_t clampi(int32_t v, int32_t lo, int32_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int32_t owner_of(float px, float py, float pz, int32_t B, int32_t nb)
{
    const int32_t bx = clampi((int32_t)floorf(px / (float)B), 0, nb - 1);
    const int32_t by = clampi((int32_t)floorf(py / (float)B), 0, nb - 1);
    const int32_t bz = clampi((int32_t)floorf(pz / (float)B), 0, nb - 1);
    return bx + nb * (by + nb * bz);
}

// Trilinear taps at p: global clamped indices g0/g1, the unclamped lower
// corner along x and y (lo), and fractions f.
struct Taps {
    int32_t g0[3], g1[3];
    int32_t lo[2];
    float f[3];
};

__device__ __forceinline__ Taps taps_at(float px, float py, float pz, int32_t N)
{
    Taps t;
    const float u[3] = {px - 0.5f, py - 0.5f, pz - 0.5f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float fl = floorf(u[a]);
        t.f[a] = u[a] - fl;
        const int32_t lo = (int32_t)fl;
        t.g0[a] = clampi(lo, 0, N - 1);
        t.g1[a] = clampi(lo + 1, 0, N - 1);
        if (a < 2) t.lo[a] = lo;
    }
    return t;
}

// sigma from the brick of x-y quads with halo 1 whose halo origin is org
// (same corners and operation order as the unpartitioned grid: a sample the
// rank owns lies within its brick, so the indices stay inside the halo)
__device__ __forceinline__ float sigma_at(const float4 *__restrict__ brick, int32_t S, const int32_t org[3],
                                          const Taps &t)
{
    const int32_t jx = clampi(t.lo[0] - org[0], 0, S - 1), jy = clampi(t.lo[1] - org[1], 0, S - 1);
    const int32_t z0 = clampi(t.g0[2] - org[2], 0, S - 1), z1 = clampi(t.g1[2] - org[2], 0, S - 1);
    return quad_trilinear(brick, S, jx, jy, z0, z1, t.f);
}

// Per-ray gradient accumulator: consecutive samples of a ray (half a voxel
// apart) mostly share their eight trilinear corners, so their weighted
// gradients are summed in registers while the corners stay the same and
// added to the grid (atomic adds) when they change or the ray leaves.
struct GradAcc {
    int32_t g0[3], g1[3];
    float v[8];
    bool any;
};

__device__ __forceinline__ void grad_flush(float *grad, int32_t N, GradAcc &A)
{
    if (!A.any) return;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int32_t ix = (c & 1) ? A.g1[0] : A.g0[0];
        const int32_t iy = (c & 2) ? A.g1[1] : A.g0[1];
        const int32_t iz = (c & 4) ? A.g1[2] : A.g0[2];
        if (A.v[c] != 0.0f) atomicAdd(grad + ((size_t)iz * N + iy) * N + ix, A.v[c]);
    }
    A.any = false;
}

__device__ __forceinline__ void grad_add(float *grad, int32_t N, GradAcc &A, const Taps &t, float gs)
{
    const bool same = A.any && A.g0[0] == t.g0[0] && A.g0[1] == t.g0[1] && A.g0[2] == t.g0[2] &&
                      A.g1[0] == t.g1[0] && A.g1[1] == t.g1[1] && A.g1[2] == t.g1[2];
    if (!same) {
        grad_flush(grad, N, A);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            A.g0[a] = t.g0[a];
            A.g1[a] = t.g1[a];
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) A.v[c] = 0.0f;
        A.any = true;
    }
    const float gx = 1.0f - t.f[0], gy = 1.0f - t.f[1], gz = 1.0f - t.f[2];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float w = ((c & 1) ? t.f[0] : gx) * ((c & 2) ? t.f[1] : gy) * ((c & 4) ? t.f[2] : gz);
        A.v[c] = A.v[c] + gs * w;
    }
}

// Primary sample s of pixel pix: 1 if it has a sample in the grid.
__device__ __forceinline__ bool make_ray(const Cam &cam, const EAParams &P, int32_t pix, int32_t s, EARay &r)
{
    const int32_t x = pix % P.W, y = pix / P.W;
    const uint4 q = philox4x32_10(make_uint4((uint32_t)pix, (uint32_t)s, 0u, 0u), make_uint2(P.seed, 5u));
    const float px = (float)x + u24(q.x), py = (float)y + u24(q.y);
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
    r.t0 = fmaxf(fmaxf(fmaxf(tn[0], tn[1]), tn[2]), 0.0f);
    r.t1 = fminf(fminf(tf[0], tf[1]), tf[2]);
    r.ox = cam.eye[0];
    r.oy = cam.eye[1];
    r.oz = cam.eye[2];
    r.dx = d[0];
    r.dy = d[1];
    r.dz = d[2];
    r.k = 0.0f;
    r.T = 1.0f;
    r.acc = 0.0f;
    r.id = (uint32_t)(pix * P.spp + s);
    r.cfin = 0.0f;
    r.g = 0.0f;
    r.lo = 0u;
    const float tk = r.t0 + 0.5f * 0.5f;
    r.rank = owner_of(r.ox + r.dx * tk, r.oy + r.dy * tk, r.oz + r.dz * tk, P.B, P.nb);
    return tk < r.t1;
}

template <bool ADJ>
__global__ void __launch_bounds__(kBlock) raygen_kernel(Cam cam, EAParams P, rf_device_queues q)
{
    const int32_t nrays = P.W * P.H * P.spp;
    for (int32_t i = blockIdx.x * kBlock + threadIdx.x; i < nrays; i += gridDim.x * kBlock) {
        const int32_t pix = i / P.spp, s = i % P.spp;
        EARay r;
        const bool hit = make_ray(cam, P, pix, s, r);
        if (!ADJ && !hit) P.rayC[i] = 0.0f;
        if (!hit) continue;
        if (ADJ) {
            r.cfin = P.rayC[i];
            r.acc = r.cfin;  // the whole suffix before the first sample
            r.lo = __float_as_uint(P.rayCLo ? P.rayCLo[i] : 0.0f);
            r.g = P.gimg[pix] / (float)P.spp;
        }
        rf::forward(q, r, r.rank);
    }
}

// ADJ: adjoint rays.  COMP (forward): keep the low part of C and return it in rayCLo.
template <bool ADJ, bool COMP>
__global__ void __launch_bounds__(kBlock) march_kernel(EAParams P, rf_device_queues q)
{
    __shared__ uint32_t sOff[RF_MAX_RANKS + 1];
    const int32_t R = q.numRanks;
    for (int e = threadIdx.x; e <= R; e += kBlock) sOff[e] = q.inOffset[e];
    __syncthreads();
    const uint32_t n = sOff[R];
    const int32_t S = P.B + 2;
    for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
        const int32_t rank = rf::rankOf(sOff, R, i);
        EARay r = rf::getIncoming<EARay>(q, i);
        const int32_t bx = rank % P.nb, by = (rank / P.nb) % P.nb, bz = rank / (P.nb * P.nb);
        const int32_t org[3] = {bx * P.B - 1, by * P.B - 1, bz * P.B - 1};
        const float4 *brick = reinterpret_cast<const float4 *>(P.bricks) + (size_t)rank * S * S * S;
        int32_t k = (int32_t)r.k;
        float T = r.T, acc = r.acc, lo = __uint_as_float(r.lo);
        GradAcc ga;
        ga.any = false;
        for (;;) {
            const float tk = r.t0 + ((float)k + 0.5f) * 0.5f;
            if (!(tk < r.t1)) {
                if (!ADJ) P.rayC[r.id] = acc;
                if (!ADJ && COMP) P.rayCLo[r.id] = lo;
                if (ADJ) grad_flush(P.grad, P.N, ga);
                break;
            }
            const float px = r.ox + r.dx * tk, py = r.oy + r.dy * tk, pz = r.oz + r.dz * tk;
            const int32_t own = owner_of(px, py, pz, P.B, P.nb);
            if (own != rank) {
                if (ADJ) grad_flush(P.grad, P.N, ga);
                r.k = (float)k;
                r.T = T;
                r.acc = acc;
                r.lo = __float_as_uint(lo);
                r.rank = own;
                rf::forward(q, r, own);
                break;
            }
            const Taps tp = taps_at(px, py, pz, P.N);
            const float sg = sigma_at(brick, S, org, tp);
            const float e = expf(-(sg * 0.5f));
            const float al = 1.0f - e;
            const float cc = sg * 20.0f;
            const float contrib = (T * al) * cc;
            if (ADJ) {
                // suffix over the later samples: (acc, lo) minus this term
                float err;
                acc = two_sum(acc, -contrib, err);
                lo = lo + err;
                const float suffix = acc + lo;
                // alpha in the derivative from expm1f: where sigma is tiny, 1 - e
                // rounds to 0 and would drop the alpha * 20 term, half of dC/dsigma
                const float alD = -expm1f(-(sg * 0.5f));
                const float dC = T * ((0.5f * e) * cc + alD * 20.0f) - 0.5f * suffix;
                grad_add(P.grad, P.N, ga, tp, r.g * dC);
            } else if (COMP) {
                float err;
                acc = two_sum(acc, contrib, err);
                lo = lo + err;
            } else {
                acc = acc + contrib;
            }
            T = T * e;
            ++k;
        }
    }
}

__global__ void __launch_bounds__(kBlock) image_kernel(const float *__restrict__ rayC, int32_t npix, int32_t spp,
                                                       float *image)
{
    for (int32_t p = blockIdx.x * kBlock + threadIdx.x; p < npix; p += gridDim.x * kBlock) {
        float sum = 0.0f;
        for (int32_t s = 0; s < spp; ++s) sum = sum + rayC[(size_t)p * spp + s];
        image[p] = sum / (float)spp;
    }
}

rf_status check_c3(rf_ctx *ctx, int32_t N, int32_t B, int32_t W, int32_t H, int32_t spp, const char *fn)
{
    if (!ctx) {
        set_error("%s: NULL context", fn);
        return RF_ERR_ARG;
    }
    if (ctx->itemBytes != sizeof(EARay)) {
        set_error("%s: rays are %zu bytes (context has %u)", fn, sizeof(EARay), ctx->itemBytes);
        return RF_ERR_ARG;
    }
    if (N < 1 || B < 1 || N % B || (int64_t)(N / B) * (N / B) * (N / B) != ctx->numRanks) {
        set_error("%s: N %d, brick %d do not give %d ranks", fn, N, B, ctx->numRanks);
        return RF_ERR_ARG;
    }
    if (W < 1 || H < 1 || spp < 1 || (uint64_t)W * H * spp > ctx->capacity) {
        set_error("%s: %d x %d x %d rays exceed the capacity", fn, W, H, spp);
        return RF_ERR_ARG;
    }
    return RF_OK;
}

Cam make_cam(const float *cam)
{
    Cam c;
    for (int a = 0; a < 3; ++a) {
        c.eye[a] = cam[a];
        c.corner[a] = cam[3 + a];
        c.du[a] = cam[6 + a];
        c.dv[a] = cam[9 + a];
    }
    return c;
}

int grid_for(rf_ctx *ctx, uint64_t work)
{
    const uint64_t want = (work + kBlock - 1) / kBlock;
    const uint64_t cap = (uint64_t)ctx->numSMs * 8u;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

template <bool ADJ>
rf_status run_ea(rf_ctx *ctx, const float *bricks, const float *cam, int32_t N, int32_t B, int32_t W, int32_t H,
                 int32_t spp, uint32_t seed, float *rayC, float *rayCLo, const float *gimg, float *grad,
                 uint32_t maxRounds, void *stream, uint64_t *rounds)
{
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    EAParams P;
    P.bricks = bricks;
    P.N = N;
    P.B = B;
    P.nb = N / B;
    P.W = W;
    P.H = H;
    P.spp = spp;
    P.seed = seed;
    P.rayC = rayC;
    P.rayCLo = rayCLo;
    P.grad = grad;
    P.gimg = gimg;
    rf_device_queues q;
    rf_get_device_queues(ctx, &q);
    const uint64_t nrays = (uint64_t)W * H * spp;
    raygen_kernel<ADJ><<<grid_for(ctx, nrays), kBlock, 0, s>>>(make_cam(cam), P, q);
    RF_LAUNCHED("c3 raygen_kernel");
    uint64_t active = 0, r = 0;
    rf_status st = rf_exchange(ctx, stream, &active);
    if (st != RF_OK) return st;
    while (active > 0) {
        if (r >= maxRounds) {
            set_error("%llu rays still active after %u rounds", (unsigned long long)active, maxRounds);
            if (rounds) *rounds = r;
            return RF_ERR_MAX_ROUNDS;
        }
        time_begin(ctx, kTimeWork, s);
        if (ADJ || !P.rayCLo) march_kernel<ADJ, false><<<grid_for(ctx, ctx->capacity), kBlock, 0, s>>>(P, q);
        else march_kernel<false, true><<<grid_for(ctx, ctx->capacity), kBlock, 0, s>>>(P, q);
        RF_LAUNCHED("c3 march_kernel");
        time_end(ctx, kTimeWork, s);
        if ((st = rf_exchange(ctx, stream, &active))) return st;
        ++r;
    }
    if (rounds) *rounds = r;
    return RF_OK;
}

}  // namespace
}  // namespace rfi

using namespace rfi;

extern "C" {

rf_status rf_c3_render(rf_ctx *ctx, const float *bricks, const float *cam, int32_t N, int32_t B, int32_t W, int32_t H,
                       int32_t spp, uint32_t seed, float *rayC, float *rayCLo, float *image, uint32_t maxRounds,
                       void *stream, uint64_t *rounds)
{
    if (rf_status st = check_c3(ctx, N, B, W, H, spp, "rf_c3_render")) return st;
    if (!bricks || !cam || !rayC || !image || (reinterpret_cast<uintptr_t>(bricks) & 15u)) {
        set_error("rf_c3_render: NULL buffer");
        return RF_ERR_ARG;
    }
    rf_status st = run_ea<false>(ctx, bricks, cam, N, B, W, H, spp, seed, rayC, rayCLo, nullptr, nullptr, maxRounds,
                                 stream, rounds);
    if (st != RF_OK) return st;
    DeviceGuard g(ctx->device);
    image_kernel<<<grid_for(ctx, (uint64_t)W * H), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(rayC, W * H, spp,
                                                                                                    image);
    RF_LAUNCHED("c3 image_kernel");
    return RF_OK;
}

rf_status rf_c3_adjoint(rf_ctx *ctx, const float *bricks, const float *cam, int32_t N, int32_t B, int32_t W,
                        int32_t H, int32_t spp, uint32_t seed, const float *rayC, const float *rayCLo,
                        const float *gradImage, float *gradVolume, uint32_t maxRounds, void *stream,
                        uint64_t *rounds)
{
    if (rf_status st = check_c3(ctx, N, B, W, H, spp, "rf_c3_adjoint")) return st;
    if (!bricks || !cam || !rayC || !gradImage || !gradVolume || (reinterpret_cast<uintptr_t>(bricks) & 15u)) {
        set_error("rf_c3_adjoint: NULL buffer");
        return RF_ERR_ARG;
    }
    return run_ea<true>(ctx, bricks, cam, N, B, W, H, spp, seed, const_cast<float *>(rayC),
                        const_cast<float *>(rayCLo), gradImage, gradVolume, maxRounds, stream, rounds);
}

}  // extern "C"
