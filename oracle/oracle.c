/*
 * Oracle for the RaFI work-forwarding hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library, its
 * Python binding) may link, load or call this file; only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark do.  It is a plain,
 * slow, single-threaded restatement of what the method computes, written
 * from the paper and the workload definitions, and it shares no code with
 * the GPU path.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared  (no FMA
 * contraction: float results of the marching workload must follow the
 * written operation order exactly).
 *
 * Contents
 *   or_philox4x32_10   counter-based generator (Salmon et al., SC'11, "Parallel
 *                      random numbers: as easy as 1, 2, 3", Philox-4x32, 10 rounds)
 *   or_partition       forwardRays' exchange result (Sec. 4.2.1 + 4.2.2): a
 *                      stable partition of the emitted items by destination
 *   or_zipf_thresholds Zipf(s) destination table for the microbenchmark
 *   or_c1_*            the forwarding microbenchmark (hop simulator)
 *   or_c0_*            absorption marching through a density grid (the VoPaT
 *                      style trace kernel of Sec. 5.1, absorption only)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10.  One round maps counter (c0,c1,c2,c3) with key (k0,k1) to */
/* (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0)); the key is     */
/* bumped by the Weyl constants between rounds.                             */
/* ------------------------------------------------------------------------ */
#define OR_PHILOX_M0 0xD2511F53u
#define OR_PHILOX_M1 0xCD9E8D57u
#define OR_PHILOX_W0 0x9E3779B9u
#define OR_PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += OR_PHILOX_W0;
            k1 += OR_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* n independent evaluations: ctr is n x 4, key is n x 2, out is n x 4. */
void or_philox_batch(uint64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    for (uint64_t i = 0; i < n; ++i)
        or_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

/* ------------------------------------------------------------------------ */
/* Exchange (Sec. 4.2.1 "Sorting by Destination", Sec. 4.2.2 "Exchanging    */
/* Rays", Sec. 4.2.3 "Wrap-up").                                            */
/*                                                                          */
/* The paper radix-sorts 64-bit keys (dest << 32 | i) and gathers the items */
/* in key order, so items end up grouped by destination and, within one     */
/* destination, in emission order: a stable partition by destination.  The */
/* per-destination begin/end scan and the Alltoall/Alltoallv steps then     */
/* hand rank r the block of items addressed to it.  On one device the       */
/* concatenation of those blocks, in rank order, is the next round's input  */
/* queue; rank r's incoming segment is [offset[r], offset[r+1]).  The total */
/* is the reduce-add of received counts (Sec. 4.2.3).                       */
/*                                                                          */
/* Written out as a counting sort.  dest == -1 marks an empty slot (the     */
/* paper's first single-array design, Sec. 3.2) and is skipped; any other   */
/* destination outside [0, R) is not a valid rank (Sec. 3.3) and is counted */
/* in *bad and dropped.                                                     */
/* Returns the number of items delivered (offset[R]).                       */
/* ------------------------------------------------------------------------ */
uint64_t or_partition(const void *items, const int32_t *dest, uint64_t n, uint32_t itemBytes,
                      int32_t R, void *out, uint64_t *offset, uint64_t *bad, uint64_t *holes)
{
    uint64_t *count = (uint64_t *)calloc((size_t)R, sizeof(uint64_t));
    uint64_t nbad = 0, nholes = 0;
    for (uint64_t i = 0; i < n; ++i) {
        int32_t d = dest[i];
        if (d == -1) nholes++;
        else if (d < 0 || d >= R) nbad++;
        else count[d]++;
    }
    /* exclusive scan of the per-destination counts */
    uint64_t run = 0;
    for (int32_t d = 0; d < R; ++d) {
        offset[d] = run;
        run += count[d];
    }
    offset[R] = run;
    /* stable placement, in emission order */
    uint64_t *next = (uint64_t *)malloc((size_t)R * sizeof(uint64_t));
    for (int32_t d = 0; d < R; ++d) next[d] = offset[d];
    const unsigned char *src = (const unsigned char *)items;
    unsigned char *dst = (unsigned char *)out;
    for (uint64_t i = 0; i < n; ++i) {
        int32_t d = dest[i];
        if (d < 0 || d >= R) continue;
        memcpy(dst + next[d] * itemBytes, src + i * itemBytes, itemBytes);
        next[d]++;
    }
    free(next);
    free(count);
    if (bad) *bad = nbad;
    if (holes) *holes = nholes;
    return run;
}

/* ------------------------------------------------------------------------ */
/* Forwarding microbenchmark (the synthetic 64-byte work item workload).    */
/*                                                                          */
/* Item: 16 uint32 words w[0..15].  Round k (k = number of hops made so     */
/* far) draws  r = Philox4x32-10(key = {seed, 1}, ctr = {w0, w1, w15, k}).  */
/*   r0 < RETIRE_THRESHOLD (= ceil(0.1 * 2^32)): the item retires as is.   */
/*   otherwise it picks a destination d from r1 (uniform, Zipf or one of    */
/*   the 6 torus neighbours of its current rank), then sets w14 = d,        */
/*   w13 ^= r2, w15 += 1 and is forwarded to rank d.                        */
/* Item i starts on rank i mod R.                                           */
/* ------------------------------------------------------------------------ */
#define OR_C1_RETIRE_THRESHOLD 429496730u
enum { OR_C1_UNIFORM = 0, OR_C1_ZIPF = 1, OR_C1_NBR6 = 2 };

/* thr[k] = floor(2^32 * P(rank <= k)) for k = 0 .. R-2, where rank k has
 * weight (k+1)^-s.  Sums run in double, in increasing j. */
void or_zipf_thresholds(int32_t R, double s, uint32_t *thr)
{
    double total = 0.0;
    for (int32_t j = 1; j <= R; ++j) total += pow((double)j, -s);
    double partial = 0.0;
    for (int32_t k = 0; k + 1 < R; ++k) {
        partial += pow((double)(k + 1), -s);
        double cdf = partial / total;
        thr[k] = (uint32_t)floor(cdf * 4294967296.0);
    }
}

int32_t or_c1_choose_dest(int32_t mode, int32_t src, uint32_t r1, int32_t R, const int32_t *grid,
                          const uint32_t *thr)
{
    if (mode == OR_C1_UNIFORM) {
        return (int32_t)(((uint64_t)r1 * (uint64_t)R) >> 32);
    }
    if (mode == OR_C1_ZIPF) {
        for (int32_t k = 0; k + 1 < R; ++k)
            if (r1 < thr[k]) return k;
        return R - 1;
    }
    /* 6-neighbour torus: rank = x + gx*(y + gy*z) */
    int32_t gx = grid[0], gy = grid[1], gz = grid[2];
    int32_t x = src % gx, y = (src / gx) % gy, z = src / (gx * gy);
    int32_t k = (int32_t)(((uint64_t)r1 * 6u) >> 32);
    switch (k) {
    case 0: x = (x + 1) % gx; break;
    case 1: x = (x + gx - 1) % gx; break;
    case 2: y = (y + 1) % gy; break;
    case 3: y = (y + gy - 1) % gy; break;
    case 4: z = (z + 1) % gz; break;
    default: z = (z + gz - 1) % gz; break;
    }
    return x + gx * (y + gy * z);
}

/* One hop of one item.  Returns 1 when the item retires (w unchanged),
 * 0 when it is forwarded (w updated, *dst set). */
int32_t or_c1_hop(uint32_t *w, uint32_t seed, uint32_t hop, int32_t src, int32_t mode, int32_t R,
                  const int32_t *grid, const uint32_t *thr, int32_t *dst)
{
    uint32_t ctr[4] = {w[0], w[1], w[15], hop};
    uint32_t key[2] = {seed, 1u};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    if (r[0] < OR_C1_RETIRE_THRESHOLD) return 1;
    int32_t d = or_c1_choose_dest(mode, src, r[1], R, grid, thr);
    w[14] = (uint32_t)d;
    w[13] ^= r[2];
    w[15] += 1u;
    *dst = d;
    return 0;
}

/* Walk every item independently until it retires (or maxHops hops).
 * Item i starts on startRank[i], or on rank i mod R when startRank is NULL.
 * final[i] = item i's payload at retirement, hops[i] = hops it made,
 * visits (optional, n x maxHops) = ranks it was forwarded to.
 * Returns the number of items that hit maxHops without retiring. */
uint64_t or_c1_walk(const uint32_t *items, uint64_t n, int32_t R, uint32_t seed, int32_t mode,
                    const int32_t *grid, const uint32_t *thr, uint32_t maxHops, const int32_t *startRank,
                    uint32_t *final, uint32_t *hops, int32_t *visits)
{
    uint64_t unfinished = 0;
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t w[16];
        memcpy(w, items + 16 * i, sizeof w);
        int32_t rank = startRank ? startRank[i] : (int32_t)(i % (uint64_t)R);
        uint32_t h = 0;
        for (;;) {
            if (h >= maxHops) { unfinished++; break; }
            int32_t d = -1;
            if (or_c1_hop(w, seed, h, rank, mode, R, grid, thr, &d)) break;
            if (visits) visits[i * maxHops + h] = d;
            rank = d;
            h++;
        }
        memcpy(final + 16 * i, w, sizeof w);
        hops[i] = h;
    }
    return unfinished;
}

/* The same workload run round by round through per-rank queues, the way
 * the forwarding layer runs it: seed (item i forwarded to rank i mod R),
 * exchange, then { every rank processes its incoming segment in order,
 * emitting in that order; exchange } until nothing is active.
 *
 * active[k]  = items in the incoming queues of round k (k = 0 .. rounds-1),
 *              active[rounds] = 0,
 * retired[k] = items that retired in round k,
 * retiredOut = payloads in retirement order (n x 16),
 * dumpItems/dumpOffsets (optional) = the incoming queue and segment offsets
 *              at the start of round dumpRound.
 * Returns the number of rounds run, or -1 if maxRounds was reached. */
int32_t or_c1_rounds(const uint32_t *items, uint64_t n, int32_t R, uint32_t seed, int32_t mode,
                     const int32_t *grid, const uint32_t *thr, uint32_t maxRounds, uint64_t *active,
                     uint64_t *retired, uint32_t *retiredOut, int32_t dumpRound, uint32_t *dumpItems,
                     uint64_t *dumpOffsets)
{
    const uint32_t itemBytes = 64;
    uint32_t *outq = (uint32_t *)malloc((size_t)(n ? n : 1) * itemBytes);
    uint32_t *inq = (uint32_t *)malloc((size_t)(n ? n : 1) * itemBytes);
    int32_t *dest = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    uint64_t *off = (uint64_t *)malloc((size_t)(R + 1) * sizeof(uint64_t));
    uint64_t nret = 0;

    /* seed round */
    memcpy(outq, items, (size_t)n * itemBytes);
    for (uint64_t i = 0; i < n; ++i) dest[i] = (int32_t)(i % (uint64_t)R);
    uint64_t nin = or_partition(outq, dest, n, itemBytes, R, inq, off, NULL, NULL);

    int32_t round = 0;
    for (;;) {
        if (round == dumpRound && dumpItems) {
            memcpy(dumpItems, inq, (size_t)nin * itemBytes);
            memcpy(dumpOffsets, off, (size_t)(R + 1) * sizeof(uint64_t));
        }
        if (nin == 0) {
            active[round] = 0;
            break;
        }
        if ((uint32_t)round >= maxRounds) {
            round = -1;
            break;
        }
        active[round] = nin;
        uint64_t nout = 0, nr = 0;
        for (int32_t r = 0; r < R; ++r) {
            for (uint64_t i = off[r]; i < off[r + 1]; ++i) {
                uint32_t w[16];
                memcpy(w, inq + 16 * i, sizeof w);
                int32_t d = -1;
                if (or_c1_hop(w, seed, (uint32_t)round, r, mode, R, grid, thr, &d)) {
                    memcpy(retiredOut + 16 * nret, w, sizeof w);
                    nret++;
                    nr++;
                } else {
                    memcpy(outq + 16 * nout, w, sizeof w);
                    dest[nout] = d;
                    nout++;
                }
            }
        }
        retired[round] = nr;
        nin = or_partition(outq, dest, nout, itemBytes, R, inq, off, NULL, NULL);
        round++;
    }
    free(outq);
    free(inq);
    free(dest);
    free(off);
    return round;
}

/* ------------------------------------------------------------------------ */
/* Absorption marching through a float density grid (the trace step of     */
/* Sec. 5.1 / Fig. 1, absorption only, fixed step).                         */
/*                                                                          */
/* Volume: N^3 floats, voxel v has centre v + 0.5, stored x fastest.        */
/* sigma(p): trilinear over voxel centres, clamp to edge.                   */
/* Camera: cam = {eye[3], corner[3], du[3], dv[3]}; the unnormalised        */
/* direction of pixel (x, y) is corner + du*(x+0.5) + dv*(y+0.5), then      */
/* divided by its length.                                                   */
/* Ray/box: slab test against [0, N]^3 gives [t0, t1].  Samples at          */
/* t_k = t0 + (k + 0.5) * 0.5 while t_k < t1, position p_k = eye + dir*t_k. */
/* tau = sum_k sigma(p_k) * 0.5 in k order; T = expf(-tau).                 */
/* A ray with no sample (no hit, or t_0 >= t1) has T = 1.                   */
/*                                                                          */
/* The owner of p is the brick (floor(p/B) clamped to the brick grid), with */
/* rank = bx + nb*(by + nb*bz).  The hop sequence of a ray is the sequence  */
/* of owners of p_0, p_1, ... with repeats collapsed: the ranks a ray must  */
/* visit when each rank holds one brick.                                    */
/* All float arithmetic is written in evaluation order, no contraction.     */
/* ------------------------------------------------------------------------ */
static float or_c0_sample(const float *vol, int32_t N, float px, float py, float pz)
{
    float u[3] = {px - 0.5f, py - 0.5f, pz - 0.5f};
    int32_t i0[3], i1[3];
    float f[3];
    for (int a = 0; a < 3; ++a) {
        float fl = floorf(u[a]);
        f[a] = u[a] - fl;
        int32_t lo = (int32_t)fl;
        int32_t hi = lo + 1;
        i0[a] = lo < 0 ? 0 : (lo > N - 1 ? N - 1 : lo);
        i1[a] = hi < 0 ? 0 : (hi > N - 1 ? N - 1 : hi);
    }
#define V(x, y, z) vol[((size_t)(z) * (size_t)N + (size_t)(y)) * (size_t)N + (size_t)(x)]
    float gx = 1.0f - f[0], gy = 1.0f - f[1], gz = 1.0f - f[2];
    float c00 = V(i0[0], i0[1], i0[2]) * gx + V(i1[0], i0[1], i0[2]) * f[0];
    float c10 = V(i0[0], i1[1], i0[2]) * gx + V(i1[0], i1[1], i0[2]) * f[0];
    float c01 = V(i0[0], i0[1], i1[2]) * gx + V(i1[0], i0[1], i1[2]) * f[0];
    float c11 = V(i0[0], i1[1], i1[2]) * gx + V(i1[0], i1[1], i1[2]) * f[0];
#undef V
    float c0 = c00 * gy + c10 * f[1];
    float c1 = c01 * gy + c11 * f[1];
    return c0 * gz + c1 * f[2];
}

static int32_t or_c0_owner(float px, float py, float pz, int32_t B, int32_t nb)
{
    float p[3] = {px, py, pz};
    int32_t b[3];
    for (int a = 0; a < 3; ++a) {
        int32_t v = (int32_t)floorf(p[a] / (float)B);
        b[a] = v < 0 ? 0 : (v > nb - 1 ? nb - 1 : v);
    }
    return b[0] + nb * (b[1] + nb * b[2]);
}

/* Primary ray of pixel (x, y): direction and [t0, t1].  Returns 1 if the
 * ray has at least one sample (t_0 < t1). */
int32_t or_c0_primary(const float *cam, int32_t N, int32_t x, int32_t y, float *dir, float *t0out,
                      float *t1out)
{
    float px = (float)x + 0.5f, py = (float)y + 0.5f;
    float d[3];
    for (int a = 0; a < 3; ++a) d[a] = cam[3 + a] + cam[6 + a] * px + cam[9 + a] * py;
    float len = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int a = 0; a < 3; ++a) d[a] = d[a] / len;
    float tn[3], tf[3];
    for (int a = 0; a < 3; ++a) {
        float ta = (0.0f - cam[a]) / d[a];
        float tb = ((float)N - cam[a]) / d[a];
        tn[a] = fminf(ta, tb);
        tf[a] = fmaxf(ta, tb);
    }
    float t0 = fmaxf(fmaxf(fmaxf(tn[0], tn[1]), tn[2]), 0.0f);
    float t1 = fminf(fminf(tf[0], tf[1]), tf[2]);
    for (int a = 0; a < 3; ++a) dir[a] = d[a];
    *t0out = t0;
    *t1out = t1;
    float tk = t0 + (0.0f + 0.5f) * 0.5f;
    return tk < t1 ? 1 : 0;
}

/* Render W x H pixels through the unpartitioned volume.
 * T[pix], tau[pix], nsamp[pix]; hop sequences for brick size B (N % B == 0)
 * into hopSeq[pix * maxHops + j], hopCount[pix] (may exceed maxHops; only
 * the first maxHops entries are stored). */
void or_c0_render(const float *vol, int32_t N, int32_t B, const float *cam, int32_t W, int32_t H,
                  float *T, float *tau, int32_t *nsamp, int32_t *hopSeq, int32_t maxHops,
                  int32_t *hopCount)
{
    int32_t nb = N / B;
    for (int32_t y = 0; y < H; ++y) {
        for (int32_t x = 0; x < W; ++x) {
            int32_t pix = y * W + x;
            float dir[3], t0, t1;
            int32_t hit = or_c0_primary(cam, N, x, y, dir, &t0, &t1);
            float acc = 0.0f;
            int32_t k = 0, hops = 0, last = -1;
            if (hit) {
                for (;;) {
                    float tk = t0 + ((float)k + 0.5f) * 0.5f;
                    if (!(tk < t1)) break;
                    float px = cam[0] + dir[0] * tk;
                    float py = cam[1] + dir[1] * tk;
                    float pz = cam[2] + dir[2] * tk;
                    int32_t own = or_c0_owner(px, py, pz, B, nb);
                    if (own != last) {
                        if (hopSeq && hops < maxHops) hopSeq[(size_t)pix * maxHops + hops] = own;
                        hops++;
                        last = own;
                    }
                    acc = acc + or_c0_sample(vol, N, px, py, pz) * 0.5f;
                    k++;
                }
            }
            tau[pix] = acc;
            T[pix] = expf(-acc);
            nsamp[pix] = k;
            if (hopCount) hopCount[pix] = hops;
        }
    }
}

/* Single-point access to sigma(p), for tests. */
float or_c0_sigma(const float *vol, int32_t N, float px, float py, float pz)
{
    return or_c0_sample(vol, N, px, py, pz);
}

/* ------------------------------------------------------------------------ */
/* Streamlines (Sec. 5.4): particles advected by RK4 through a trilinear     */
/* vector field, one particle per work item, forwarded between the ranks     */
/* that own the grid's bricks.                                               */
/*                                                                          */
/* field: N^3 x 3 floats, index ((z*N + y)*N + x)*3 + c, voxel centres at    */
/* v + 0.5.  v(p): trilinear per component over voxel centres, clamp to      */
/* edge (the weights of the marching workload).                             */
/* One step (float, written order, no contraction), step h:                 */
/*   k1 = v(p); k2 = v(p + (h*0.5)*k1); k3 = v(p + (h*0.5)*k2);             */
/*   k4 = v(p + h*k3); p' = p + (h/6)*(((k1 + 2*k2) + 2*k3) + k4)           */
/* A particle stops when it has made maxSteps steps (status 3), when a step */
/* does not move it (p' == p, status 2), or when p' leaves [0, N)^3 (the    */
/* step is taken, status 1).  hops = changes of owner brick (brick B) along */
/* the accepted positions inside the grid.                                  */
/* ------------------------------------------------------------------------ */
static void or_c2_sample(const float *f, int32_t N, const float *p, float *out)
{
    int32_t i0[3], i1[3];
    float fr[3];
    for (int a = 0; a < 3; ++a) {
        float u = p[a] - 0.5f;
        float fl = floorf(u);
        fr[a] = u - fl;
        int32_t lo = (int32_t)fl;
        int32_t hi = lo + 1;
        i0[a] = lo < 0 ? 0 : (lo > N - 1 ? N - 1 : lo);
        i1[a] = hi < 0 ? 0 : (hi > N - 1 ? N - 1 : hi);
    }
    float gx = 1.0f - fr[0], gy = 1.0f - fr[1], gz = 1.0f - fr[2];
#define F(x, y, z, c) f[(((size_t)(z) * (size_t)N + (size_t)(y)) * (size_t)N + (size_t)(x)) * 3u + (c)]
    for (int c = 0; c < 3; ++c) {
        float c00 = F(i0[0], i0[1], i0[2], c) * gx + F(i1[0], i0[1], i0[2], c) * fr[0];
        float c10 = F(i0[0], i1[1], i0[2], c) * gx + F(i1[0], i1[1], i0[2], c) * fr[0];
        float c01 = F(i0[0], i0[1], i1[2], c) * gx + F(i1[0], i0[1], i1[2], c) * fr[0];
        float c11 = F(i0[0], i1[1], i1[2], c) * gx + F(i1[0], i1[1], i1[2], c) * fr[0];
        float c0 = c00 * gy + c10 * fr[1];
        float c1 = c01 * gy + c11 * fr[1];
        out[c] = c0 * gz + c1 * fr[2];
    }
#undef F
}

/* one RK4 step from p into q */
void or_c2_rk4(const float *f, int32_t N, float h, const float *p, float *q)
{
    float k1[3], k2[3], k3[3], k4[3], t[3];
    float half = h * 0.5f, sixth = h / 6.0f;
    or_c2_sample(f, N, p, k1);
    for (int a = 0; a < 3; ++a) t[a] = p[a] + half * k1[a];
    or_c2_sample(f, N, t, k2);
    for (int a = 0; a < 3; ++a) t[a] = p[a] + half * k2[a];
    or_c2_sample(f, N, t, k3);
    for (int a = 0; a < 3; ++a) t[a] = p[a] + h * k3[a];
    or_c2_sample(f, N, t, k4);
    for (int a = 0; a < 3; ++a) {
        float s = ((k1[a] + 2.0f * k2[a]) + 2.0f * k3[a]) + k4[a];
        q[a] = p[a] + sixth * s;
    }
}

/* v(p) for tests */
void or_c2_velocity(const float *f, int32_t N, const float *p, float *out) { or_c2_sample(f, N, p, out); }

/* Trace n particles through the unpartitioned field.  seeds n x 3;
 * outputs: pos n x 3 (final position), steps, hops, status. */
void or_c2_trace(const float *f, int32_t N, int32_t B, const float *seeds, uint64_t n, float h, uint32_t maxSteps,
                 float *pos, uint32_t *steps, uint32_t *hops, uint32_t *status)
{
    int32_t nb = N / B;
    for (uint64_t i = 0; i < n; ++i) {
        float p[3] = {seeds[3 * i], seeds[3 * i + 1], seeds[3 * i + 2]};
        uint32_t k = 0, hp = 0, st = 0;
        int32_t own = or_c0_owner(p[0], p[1], p[2], B, nb);
        for (;;) {
            if (k >= maxSteps) { st = 3; break; }
            float q[3];
            or_c2_rk4(f, N, h, p, q);
            if (q[0] == p[0] && q[1] == p[1] && q[2] == p[2]) { st = 2; break; }
            k++;
            p[0] = q[0]; p[1] = q[1]; p[2] = q[2];
            if (!(p[0] >= 0.0f && p[0] < (float)N && p[1] >= 0.0f && p[1] < (float)N && p[2] >= 0.0f &&
                  p[2] < (float)N)) { st = 1; break; }
            int32_t o = or_c0_owner(p[0], p[1], p[2], B, nb);
            if (o != own) { hp++; own = o; }
        }
        pos[3 * i] = p[0]; pos[3 * i + 1] = p[1]; pos[3 * i + 2] = p[2];
        steps[i] = k;
        hops[i] = hp;
        status[i] = st;
    }
}

/* ------------------------------------------------------------------------ */
/* Differentiable emission-absorption rendering through the same kind of    */
/* density grid (the Lander renderer's integration model, Sec. 5.2, on a    */
/* structured grid).                                                        */
/*                                                                          */
/* spp jittered primary rays per pixel: sample s of pixel p = y*W + x       */
/* aims at (x + u, y + v), u = hi24(r0) / 2^24, v = hi24(r1) / 2^24 with    */
/* r = Philox4x32-10(key {seed, 5}, counter {p, s, 0, 0}).                  */
/* Samples t_k = t0 + (k + 0.5) * 0.5 while t_k < t1 (as in the marching    */
/* workload).  With sigma_k = sigma(p_k):                                   */
/*   e_k = expf(-sigma_k * 0.5), alpha_k = 1 - e_k, c_k = sigma_k * 20      */
/*   C += (T * alpha_k) * c_k;  T = T * e_k        (T starts at 1, C at 0)  */
/* The pixel value is the mean of its samples' C.                            */
/* ------------------------------------------------------------------------ */
static float or_u24(uint32_t r) { return (float)(r >> 8) * (1.0f / 16777216.0f); }

/* direction and box interval of sample s of pixel (x, y); 1 if it has a sample */
static int32_t or_c3_ray(const float *cam, int32_t N, int32_t W, int32_t x, int32_t y, int32_t s, uint32_t seed,
                         float *dir, float *t0out, float *t1out)
{
    uint32_t ctr[4] = {(uint32_t)(y * W + x), (uint32_t)s, 0u, 0u};
    uint32_t key[2] = {seed, 5u};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    float px = (float)x + or_u24(r[0]), py = (float)y + or_u24(r[1]);
    float d[3];
    for (int a = 0; a < 3; ++a) d[a] = cam[3 + a] + cam[6 + a] * px + cam[9 + a] * py;
    float len = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int a = 0; a < 3; ++a) d[a] = d[a] / len;
    float tn[3], tf[3];
    for (int a = 0; a < 3; ++a) {
        float ta = (0.0f - cam[a]) / d[a];
        float tb = ((float)N - cam[a]) / d[a];
        tn[a] = fminf(ta, tb);
        tf[a] = fmaxf(ta, tb);
    }
    float t0 = fmaxf(fmaxf(fmaxf(tn[0], tn[1]), tn[2]), 0.0f);
    float t1 = fminf(fminf(tf[0], tf[1]), tf[2]);
    for (int a = 0; a < 3; ++a) dir[a] = d[a];
    *t0out = t0;
    *t1out = t1;
    return (t0 + 0.5f * 0.5f) < t1 ? 1 : 0;
}

/* Forward render (float, written order).  rayC[(p*spp + s)] = C of each
 * sample, image[p] = their mean (sum in sample order, then / spp). */
void or_c3_render(const float *vol, int32_t N, const float *cam, int32_t W, int32_t H, int32_t spp, uint32_t seed,
                  float *rayC, float *image)
{
    for (int32_t y = 0; y < H; ++y) {
        for (int32_t x = 0; x < W; ++x) {
            int32_t pix = y * W + x;
            float sum = 0.0f;
            for (int32_t s = 0; s < spp; ++s) {
                float dir[3], t0, t1;
                float T = 1.0f, C = 0.0f;
                if (or_c3_ray(cam, N, W, x, y, s, seed, dir, &t0, &t1)) {
                    for (int32_t k = 0;; ++k) {
                        float tk = t0 + ((float)k + 0.5f) * 0.5f;
                        if (!(tk < t1)) break;
                        float px = cam[0] + dir[0] * tk, py = cam[1] + dir[1] * tk, pz = cam[2] + dir[2] * tk;
                        float sg = or_c0_sample(vol, N, px, py, pz);
                        float e = expf(-(sg * 0.5f));
                        float al = 1.0f - e;
                        float cc = sg * 20.0f;
                        C = C + (T * al) * cc;
                        T = T * e;
                    }
                }
                rayC[(size_t)pix * spp + s] = C;
                sum = sum + C;
            }
            image[pix] = sum / (float)spp;
        }
    }
}

/* Reference gradient, in double: dL/dvol given dLdC per sample ray
 * ((p*spp + s) order).  Every quantity is recomputed in double from the
 * float volume (sigma by trilinear interpolation in double, positions from
 * the float ray).  Per ray: forward to collect sigma_k, T_k, alpha_k, c_k;
 * then k from last to first with the suffix S = sum_{j>k} T_j alpha_j c_j:
 *   dC/dsigma_k = T_k (0.5 e_k c_k + alpha_k * 20) - 0.5 S,
 * scattered to the 8 voxels with the trilinear weights (clamped taps add).
 * gabs (may be NULL) receives, per voxel, the same sum taken over the
 * magnitudes of the parts, |dLdC| (|T_k (0.5 e_k c_k + alpha_k * 20)| +
 * |0.5 S|) weight: the scale against which a float evaluation and sum of the
 * contributions can be judged, since each is the difference of its two parts
 * (it is not part of the gradient).  gcount (may be NULL) receives, per
 * voxel, the number of (sample, corner) contributions added to it.
 * Returns the loss-independent sum of dLdC * C (a consistency value). */
double or_c3_adjoint_f64(const float *vol, int32_t N, const float *cam, int32_t W, int32_t H, int32_t spp,
                         uint32_t seed, const double *dLdC, double *grad, double *gabs, double *gcount)
{
    int32_t maxK = (int32_t)(2.0f * 1.7321f * (float)N) + 8;
    double *sg = (double *)malloc((size_t)maxK * sizeof(double));
    double *Tk = (double *)malloc((size_t)maxK * sizeof(double));
    float *pk = (float *)malloc((size_t)maxK * 3 * sizeof(float));
    double acc = 0.0;
    for (int32_t y = 0; y < H; ++y) {
        for (int32_t x = 0; x < W; ++x) {
            int32_t pix = y * W + x;
            for (int32_t s = 0; s < spp; ++s) {
                double g = dLdC[(size_t)pix * spp + s];
                float dir[3], t0, t1;
                if (!or_c3_ray(cam, N, W, x, y, s, seed, dir, &t0, &t1)) continue;
                int32_t K = 0;
                double T = 1.0, C = 0.0;
                for (;; ++K) {
                    float tk = t0 + ((float)K + 0.5f) * 0.5f;
                    if (!(tk < t1) || K >= maxK) break;
                    float p[3] = {cam[0] + dir[0] * tk, cam[1] + dir[1] * tk, cam[2] + dir[2] * tk};
                    /* trilinear in double */
                    double w[3];
                    int32_t i0[3], i1[3];
                    for (int a = 0; a < 3; ++a) {
                        double u = (double)p[a] - 0.5, fl = floor(u);
                        w[a] = u - fl;
                        int32_t lo = (int32_t)fl, hi = lo + 1;
                        i0[a] = lo < 0 ? 0 : (lo > N - 1 ? N - 1 : lo);
                        i1[a] = hi < 0 ? 0 : (hi > N - 1 ? N - 1 : hi);
                    }
                    double v = 0.0;
                    for (int c = 0; c < 8; ++c) {
                        int32_t ix = (c & 1) ? i1[0] : i0[0], iy = (c & 2) ? i1[1] : i0[1], iz = (c & 4) ? i1[2] : i0[2];
                        double wt = ((c & 1) ? w[0] : 1.0 - w[0]) * ((c & 2) ? w[1] : 1.0 - w[1]) *
                                    ((c & 4) ? w[2] : 1.0 - w[2]);
                        v += wt * (double)vol[((size_t)iz * N + iy) * N + ix];
                    }
                    sg[K] = v;
                    Tk[K] = T;
                    pk[3 * K] = p[0]; pk[3 * K + 1] = p[1]; pk[3 * K + 2] = p[2];
                    double e = exp(-v * 0.5);
                    C += T * (1.0 - e) * (v * 20.0);
                    T *= e;
                }
                acc += g * C;
                double S = 0.0;
                for (int32_t k = K - 1; k >= 0; --k) {
                    double e = exp(-sg[k] * 0.5), al = 1.0 - e, cc = sg[k] * 20.0;
                    double first = Tk[k] * (0.5 * e * cc + al * 20.0);
                    double dCds = first - 0.5 * S;
                    double scale = fabs(g) * (fabs(first) + 0.5 * fabs(S));
                    S += Tk[k] * al * cc;
                    double gs = g * dCds;
                    double w[3];
                    int32_t i0[3], i1[3];
                    for (int a = 0; a < 3; ++a) {
                        double u = (double)pk[3 * k + a] - 0.5, fl = floor(u);
                        w[a] = u - fl;
                        int32_t lo = (int32_t)fl, hi = lo + 1;
                        i0[a] = lo < 0 ? 0 : (lo > N - 1 ? N - 1 : lo);
                        i1[a] = hi < 0 ? 0 : (hi > N - 1 ? N - 1 : hi);
                    }
                    for (int c = 0; c < 8; ++c) {
                        int32_t ix = (c & 1) ? i1[0] : i0[0], iy = (c & 2) ? i1[1] : i0[1], iz = (c & 4) ? i1[2] : i0[2];
                        double wt = ((c & 1) ? w[0] : 1.0 - w[0]) * ((c & 2) ? w[1] : 1.0 - w[1]) *
                                    ((c & 4) ? w[2] : 1.0 - w[2]);
                        grad[((size_t)iz * N + iy) * N + ix] += gs * wt;
                        if (gabs) gabs[((size_t)iz * N + iy) * N + ix] += scale * wt;
                        if (gcount) gcount[((size_t)iz * N + iy) * N + ix] += 1.0;
                    }
                }
            }
        }
    }
    free(sg);
    free(Tk);
    free(pk);
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Stochastic transport by delta tracking (VoPaT's trace step, Sec. 5.1,    */
/* Fig. 1: rays that collide scatter and are forwarded to themselves, rays  */
/* that leave the local data go to the next rank).                         */
/*                                                                          */
/* Path (gpix, s): jittered primary ray (Philox key {seed, 9}, counter      */
/* {gpix, s, 0, 0}, as the emission-absorption renderer) enters [0,N)^3 at  */
/* t0 (a miss escapes at once).  Event (bounce b, index e): r = Philox(key  */
/* {seed, 7}, counter {gpix, s, b, e}); free flight t = -logf(1 - u(r0)) /  */
/* sigmaMax; q = p + t d.  q outside the grid: the path escapes and scores  */
/* 1 (environment radiance 1).  Otherwise with sigma(q) (trilinear): a real */
/* collision when u(r1) * sigmaMax < sigma; then u(r2) < 0.8 scatters (b+1; */
/* more than 64 bounces score 0) with a Henyey-Greenstein (g = 0.3)         */
/* direction from u(r3) and u of word 0 of Philox(key {seed, 8}, counter    */
/* {gpix, s, b, e}); otherwise the path is absorbed (scores 0).  A null     */
/* collision moves p to q and increments e.  u(r) = top 24 bits / 2^24.     */
/* ------------------------------------------------------------------------ */
static void or_c4_hg(float *d, float xi, float xphi)
{
    const float g = 0.3f;
    float s = (1.0f - g * g) / (1.0f - g + 2.0f * g * xi);
    float ct = (1.0f + g * g - s * s) / (2.0f * g);
    ct = fminf(1.0f, fmaxf(-1.0f, ct));
    float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
    float phi = 6.2831853f * xphi;
    float cp = cosf(phi), sp = sinf(phi);
    float ax = fabsf(d[0]) < 0.9f ? 1.0f : 0.0f, ay = 1.0f - ax;
    /* u = normalize(d x a), v = d x u */
    float ux = d[1] * 0.0f - d[2] * ay, uy = d[2] * ax - d[0] * 0.0f, uz = d[0] * ay - d[1] * ax;
    float ul = sqrtf(ux * ux + uy * uy + uz * uz);
    ux = ux / ul; uy = uy / ul; uz = uz / ul;
    float vx = d[1] * uz - d[2] * uy, vy = d[2] * ux - d[0] * uz, vz = d[0] * uy - d[1] * ux;
    float nx = (st * cp) * ux + (st * sp) * vx + ct * d[0];
    float ny = (st * cp) * uy + (st * sp) * vy + ct * d[1];
    float nz = (st * cp) * uz + (st * sp) * vz + ct * d[2];
    float nl = sqrtf(nx * nx + ny * ny + nz * nz);
    d[0] = nx / nl; d[1] = ny / nl; d[2] = nz / nl;
}

/* score (0 or 1) of one path; *events = events drawn, *bounces = scatterings */
int32_t or_c4_path(const float *vol, int32_t N, float sigmaMax, const float *cam, int32_t W, int32_t x, int32_t y,
                   uint32_t gpix, uint32_t s, uint32_t seed, uint32_t *events, uint32_t *bounces)
{
    uint32_t ctr[4] = {gpix, s, 0u, 0u}, key[2] = {seed, 9u}, r[4];
    or_philox4x32_10(ctr, key, r);
    float px = (float)x + or_u24(r[0]), py = (float)y + or_u24(r[1]);
    float d[3];
    for (int a = 0; a < 3; ++a) d[a] = cam[3 + a] + cam[6 + a] * px + cam[9 + a] * py;
    float len = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int a = 0; a < 3; ++a) d[a] = d[a] / len;
    float tn[3], tf[3];
    for (int a = 0; a < 3; ++a) {
        float ta = (0.0f - cam[a]) / d[a];
        float tb = ((float)N - cam[a]) / d[a];
        tn[a] = fminf(ta, tb);
        tf[a] = fmaxf(ta, tb);
    }
    float t0 = fmaxf(fmaxf(fmaxf(tn[0], tn[1]), tn[2]), 0.0f);
    float t1 = fminf(fminf(tf[0], tf[1]), tf[2]);
    *events = 0;
    *bounces = 0;
    if (!(t0 < t1)) return 1;
    float p[3] = {cam[0] + d[0] * t0, cam[1] + d[1] * t0, cam[2] + d[2] * t0};
    uint32_t b = 0, e = 0;
    for (;;) {
        uint32_t c2[4] = {gpix, s, b, e}, k2[2] = {seed, 7u}, q4[4];
        or_philox4x32_10(c2, k2, q4);
        (*events)++;
        float t = -logf(1.0f - or_u24(q4[0])) / sigmaMax;
        float q[3] = {p[0] + d[0] * t, p[1] + d[1] * t, p[2] + d[2] * t};
        if (!(q[0] >= 0.0f && q[0] < (float)N && q[1] >= 0.0f && q[1] < (float)N && q[2] >= 0.0f &&
              q[2] < (float)N))
            return 1;
        float sg = or_c0_sample(vol, N, q[0], q[1], q[2]);
        p[0] = q[0]; p[1] = q[1]; p[2] = q[2];
        if (or_u24(q4[1]) * sigmaMax < sg) {
            if (!(or_u24(q4[2]) < 0.8f)) return 0;
            uint32_t k3[2] = {seed, 8u}, h4[4];
            or_philox4x32_10(c2, k3, h4);
            b++;
            (*bounces)++;
            if (b > 64u) return 0;
            or_c4_hg(d, or_u24(q4[3]), or_u24(h4[0]));
            e = 0;
        } else {
            e++;
        }
    }
}

/* A crop [x0, x0+cw) x [y0, y0+ch) of a W x H view whose first pixel has
 * global index pixBase: image = mean score over spp paths per pixel. */
void or_c4_render_crop(const float *vol, int32_t N, float sigmaMax, const float *cam, int32_t W, uint32_t pixBase,
                       int32_t x0, int32_t y0, int32_t cw, int32_t ch, int32_t spp, uint32_t seed, float *image,
                       uint64_t *events)
{
    uint64_t ev = 0;
    for (int32_t yy = 0; yy < ch; ++yy) {
        for (int32_t xx = 0; xx < cw; ++xx) {
            int32_t x = x0 + xx, y = y0 + yy;
            uint32_t gpix = pixBase + (uint32_t)(y * W + x);
            int32_t sum = 0;
            for (int32_t s = 0; s < spp; ++s) {
                uint32_t e, b;
                sum += or_c4_path(vol, N, sigmaMax, cam, W, x, y, gpix, (uint32_t)s, seed, &e, &b);
                ev += e;
            }
            image[yy * cw + xx] = (float)sum / (float)spp;
        }
    }
    if (events) *events = ev;
}

/* test access to the Henyey-Greenstein sampler */
void or_c4_hg_sample(const float *d, float xi, float xphi, float *out)
{
    out[0] = d[0]; out[1] = d[1]; out[2] = d[2];
    or_c4_hg(out, xi, xphi);
}

/* ------------------------------------------------------------------------ */
/* Multi-phase exchange with three item types (the protocol of Sec. 5.5:    */
/* particle migration, then an essential-tree exchange in which each rank   */
/* broadcasts its root multipole node, peers that need finer data send a    */
/* refinement request back, and the owner answers with the child nodes).    */
/* Synthetic and integer-only: positions are 32-bit fixed point on the      */
/* periodic unit cube, split into a 2^lgx x 2^lgy x 2^lgz grid of ranks;    */
/* a node is the mass, the mass-weighted coordinate sums and the particle   */
/* count of one rank (the root) or of one octant of its box (a child).      */
/* ------------------------------------------------------------------------ */

/* rank owning position (x, y, z): the top lg bits of each coordinate */
int32_t or_mp_owner(uint32_t x, uint32_t y, uint32_t z, const int32_t lg[3])
{
    const uint32_t bx = lg[0] ? x >> (32 - lg[0]) : 0u;
    const uint32_t by = lg[1] ? y >> (32 - lg[1]) : 0u;
    const uint32_t bz = lg[2] ? z >> (32 - lg[2]) : 0u;
    const uint32_t gx = (uint32_t)1 << lg[0], gy = (uint32_t)1 << lg[1];
    return (int32_t)(bx + gx * (by + gy * bz));
}

/* octant of a position inside its rank's box: the bit after the rank bits */
static int32_t or_mp_octant(uint32_t x, uint32_t y, uint32_t z, const int32_t lg[3])
{
    return (int32_t)(((x >> (31 - lg[0])) & 1u) | (((y >> (31 - lg[1])) & 1u) << 1) |
                     (((z >> (31 - lg[2])) & 1u) << 2));
}

/* Particle i (8 words: x, y, z, vx, vy, vz, m, id) moves by its velocity,
 * wrapping around the periodic cube; owner[i] = rank of the new position. */
void or_mp_migrate(const uint32_t *p, uint64_t n, const int32_t lg[3], uint32_t *out, int32_t *owner)
{
    for (uint64_t i = 0; i < n; ++i) {
        const uint32_t *a = p + 8 * i;
        uint32_t *b = out + 8 * i;
        for (int k = 0; k < 8; ++k) b[k] = a[k];
        b[0] = a[0] + a[3];
        b[1] = a[1] + a[4];
        b[2] = a[2] + a[5];
        owner[i] = or_mp_owner(b[0], b[1], b[2], lg);
    }
}

/* Local trees: nodes[(r * 9 + c) * 5 + {0..4}] = {M, X, Y, Z, count} of rank
 * r's particles (c = 0, the root) and of those in octant c - 1 of its box. */
void or_mp_tree(const uint32_t *p, uint64_t n, const int32_t lg[3], uint64_t *nodes)
{
    const int32_t R = 1 << (lg[0] + lg[1] + lg[2]);
    for (int64_t k = 0; k < (int64_t)R * 9 * 5; ++k) nodes[k] = 0;
    for (uint64_t i = 0; i < n; ++i) {
        const uint32_t *a = p + 8 * i;
        const int32_t r = or_mp_owner(a[0], a[1], a[2], lg);
        const int32_t c[2] = {0, 1 + or_mp_octant(a[0], a[1], a[2], lg)};
        for (int j = 0; j < 2; ++j) {
            uint64_t *nd = nodes + ((uint64_t)r * 9 + (uint64_t)c[j]) * 5;
            nd[0] += a[6];
            nd[1] += (uint64_t)a[6] * a[0];
            nd[2] += (uint64_t)a[6] * a[1];
            nd[3] += (uint64_t)a[6] * a[2];
            nd[4] += 1;
        }
    }
}

/* 1 if rank s is one of rank r's 26 torus neighbours (Chebyshev distance 1
 * per axis with wrap-around, s != r); peers this close ask for children. */
int32_t or_mp_near(int32_t r, int32_t s, const int32_t lg[3])
{
    if (r == s) return 0;
    int32_t rc[3], sc[3];
    int32_t t = r, u = s;
    for (int k = 0; k < 3; ++k) {
        const int32_t g = 1 << lg[k];
        rc[k] = t % g;
        sc[k] = u % g;
        t /= g;
        u /= g;
    }
    for (int k = 0; k < 3; ++k) {
        const int32_t g = 1 << lg[k];
        const int32_t d = (rc[k] - sc[k] + g) % g;
        if (d != 0 && d != 1 && d != g - 1) return 0;
    }
    return 1;
}
