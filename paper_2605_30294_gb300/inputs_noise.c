/*
 * Seeded input generator: fractal gradient noise for the transport
 * workload's density grid.  Input data only (no transport arithmetic); both
 * the CUDA path and the oracle read the grid it writes.
 *
 * Gradient noise after Perlin's "Improving Noise" (SIGGRAPH 2002): a
 * seeded permutation of 0..255 hashes the integer lattice; each lattice
 * corner holds one of 12 edge-direction gradients (the 16 entries repeat
 * four of them); the value at a point blends the 8 corner dot products with
 * the quintic fade 6t^5 - 15t^4 + 10t^3.  Octave o samples the noise at
 * frequency base * 2^o with weight 2^-o.  Evaluated in double, stored as float.
 *
 * The permutation is a Fisher-Yates shuffle driven by Philox4x32-10
 * (key {seed, 10}, counter {i, 0, 0, 0} for swap i).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

static void philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1, n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* the 16 gradient directions: the 12 cube-edge midpoints, then 4 repeated */
static const double kGrad[16][3] = {{1, 1, 0},  {-1, 1, 0}, {1, -1, 0}, {-1, -1, 0}, {1, 0, 1},  {-1, 0, 1},
                                    {1, 0, -1}, {-1, 0, -1}, {0, 1, 1},  {0, -1, 1}, {0, 1, -1}, {0, -1, -1},
                                    {1, 1, 0},  {0, -1, 1}, {-1, 1, 0}, {0, -1, -1}};

static double fade(double t) { return t * t * t * (t * (t * 6.0 - 15.0) + 10.0); }

static double gnoise(const int32_t *perm, double x, double y, double z)
{
    double fx = floor(x), fy = floor(y), fz = floor(z);
    int32_t X = (int32_t)fx & 255, Y = (int32_t)fy & 255, Z = (int32_t)fz & 255;
    double rx = x - fx, ry = y - fy, rz = z - fz;
    double corner[8];
    for (int c = 0; c < 8; ++c) {
        int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        int32_t h = perm[perm[perm[(X + dx) & 255] + ((Y + dy) & 255)] + ((Z + dz) & 255)] & 15;
        corner[c] = kGrad[h][0] * (rx - dx) + kGrad[h][1] * (ry - dy) + kGrad[h][2] * (rz - dz);
    }
    double u = fade(rx), v = fade(ry), w = fade(rz);
    double x00 = corner[0] + u * (corner[1] - corner[0]);
    double x10 = corner[2] + u * (corner[3] - corner[2]);
    double x01 = corner[4] + u * (corner[5] - corner[4]);
    double x11 = corner[6] + u * (corner[7] - corner[6]);
    double y0 = x00 + v * (x10 - x00), y1 = x01 + v * (x11 - x01);
    return y0 + w * (y1 - y0);
}

static void make_perm(uint32_t seed, int32_t perm[512])
{
    int32_t p[256];
    for (int i = 0; i < 256; ++i) p[i] = i;
    for (int i = 255; i > 0; --i) {
        uint32_t ctr[4] = {(uint32_t)i, 0u, 0u, 0u}, key[2] = {seed, 10u}, r[4];
        philox(ctr, key, r);
        int j = (int)(((uint64_t)r[0] * (uint64_t)(i + 1)) >> 32);
        int t = p[i];
        p[i] = p[j];
        p[j] = t;
    }
    for (int i = 0; i < 512; ++i) perm[i] = p[i & 255];
}

/* fractal noise at voxel centres of an n^3 grid (index [z][y][x]), clamped at 0 */
void noise_volume(int32_t n, uint32_t seed, int32_t octaves, double baseFreq, float *out, double *sumOut)
{
    int32_t perm[512];
    make_perm(seed, perm);
    double total = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
    for (int32_t z = 0; z < n; ++z) {
        for (int32_t y = 0; y < n; ++y) {
            float *row = out + ((size_t)z * n + y) * n;
            for (int32_t x = 0; x < n; ++x) {
                double px = (x + 0.5) / n, py = (y + 0.5) / n, pz = (z + 0.5) / n;
                double v = 0.0, f = baseFreq, a = 1.0;
                for (int o = 0; o < octaves; ++o) {
                    v += a * gnoise(perm, px * f, py * f, pz * f);
                    f *= 2.0;
                    a *= 0.5;
                }
                float s = v > 0.0 ? (float)v : 0.0f;
                row[x] = s;
                total += (double)s;
            }
        }
    }
    *sumOut = total;
}

/* one value (tests) */
double noise_at(uint32_t seed, int32_t octaves, double baseFreq, double px, double py, double pz)
{
    int32_t perm[512];
    make_perm(seed, perm);
    double v = 0.0, f = baseFreq, a = 1.0;
    for (int o = 0; o < octaves; ++o) {
        v += a * gnoise(perm, px * f, py * f, pz * f);
        f *= 2.0;
        a *= 0.5;
    }
    return v;
}
