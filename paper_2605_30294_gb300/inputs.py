"""Seeded synthetic inputs for the forwarding workloads.

This module only makes input data (work-item payloads, density grids,
cameras); it holds none of the forwarding method's arithmetic.  Both the
CUDA path and the oracle consume what it produces.  Random words come from
Philox4x32-10 (Salmon et al., SC'11), implemented here from its published
definition in vectorised numpy.

Recipes
  microbenchmark items  item i, word 4j+m = Philox(key={seed,0}, ctr={i,j,0,0})[m]
  density grid          sum of Gaussian blobs, 0.05 * exp(-|x-c|^2 / (2 s^2)) at voxel
                        centres x = v + 0.5, evaluated in float64, stored as float32;
                        s ~ U[4,10] * (N/64), c ~ U[s, N-s]^3, uniforms from
                        Philox(key={seed,2}, ctr={blob, 0, 0, 0})
  camera                pinhole, eye/at/up/vertical fov; returns float32
                        {eye, corner, du, dv} with direction(x, y) = corner + du*(x+0.5)
                        + dv*(y+0.5) before normalisation (y = 0 is the top row)
"""
from __future__ import annotations

import math

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_LO = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10; all arguments broadcast, returns 4 uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint32) for c in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for r in range(10):
            if r:
                k0 = np.uint32((int(k0) + int(_W0)) & 0xFFFFFFFF)
                k1 = np.uint32((int(k1) + int(_W1)) & 0xFFFFFFFF)
            p0 = c0.astype(np.uint64) * _M0
            p1 = c2.astype(np.uint64) * _M1
            n0 = (p1 >> _S32).astype(np.uint32) ^ c1 ^ k0
            n1 = (p1 & _LO).astype(np.uint32)
            n2 = (p0 >> _S32).astype(np.uint32) ^ c3 ^ k1
            n3 = (p0 & _LO).astype(np.uint32)
            c0, c1, c2, c3 = n0, n1, n2, n3
    return c0, c1, c2, c3


def c1_items(n: int, seed: int = 1, chunk: int = 1 << 20) -> np.ndarray:
    """``n`` 64-byte work items (n x 16 uint32) for the forwarding microbenchmark."""
    out = np.empty((n, 16), np.uint32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        i = np.arange(s, e, dtype=np.uint32)
        z = np.zeros_like(i)
        for j in range(4):
            r = philox4x32_10(i, np.full_like(i, j), z, z, seed, 0)
            for m in range(4):
                out[s:e, 4 * j + m] = r[m]
    return out


def _uniform01(words: np.ndarray) -> np.ndarray:
    return words.astype(np.float64) / 4294967296.0


def c0_blobs(n: int = 64, nblobs: int = 8, seed: int = 0):
    """Blob centres (nblobs x 3) and widths for an n^3 grid."""
    b = np.arange(nblobs, dtype=np.uint32)
    z = np.zeros_like(b)
    r = philox4x32_10(b, z, z, z, seed, 2)
    scale = n / 64.0
    s = (4.0 + 6.0 * _uniform01(r[0])) * scale
    cen = np.stack([s + (n - 2.0 * s) * _uniform01(r[m]) for m in (1, 2, 3)], axis=1)
    return cen, s


def c0_volume(n: int = 64, nblobs: int = 8, seed: int = 0, peak: float = 0.05) -> np.ndarray:
    """n^3 float32 density, index [z, y, x] (x fastest)."""
    cen, s = c0_blobs(n, nblobs, seed)
    ax = np.arange(n, dtype=np.float64) + 0.5
    vol = np.zeros((n, n, n), np.float64)
    for zs in range(0, n, 16):
        zz = ax[zs:zs + 16][:, None, None]
        yy = ax[None, :, None]
        xx = ax[None, None, :]
        acc = np.zeros((len(ax[zs:zs + 16]), n, n), np.float64)
        for b in range(len(s)):
            d2 = (xx - cen[b, 0]) ** 2 + (yy - cen[b, 1]) ** 2 + (zz - cen[b, 2]) ** 2
            acc += peak * np.exp(-d2 / (2.0 * s[b] * s[b]))
        vol[zs:zs + 16] = acc
    return vol.astype(np.float32)


def camera(eye, at, up, fov_deg: float, width: int, height: int) -> np.ndarray:
    """Pinhole camera as float32[12] = {eye, corner, du, dv} (computed in float64)."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(at, np.float64) - eye
    f /= np.linalg.norm(f)
    upv = np.asarray(up, np.float64)
    r = np.cross(upv, f)
    r /= np.linalg.norm(r)
    u = np.cross(f, r)
    h = math.tan(math.radians(fov_deg) * 0.5)
    a = width / height
    corner = f - h * a * r + h * u
    du = (2.0 * h * a / width) * r
    dv = -(2.0 * h / height) * u
    return np.concatenate([eye, corner, du, dv]).astype(np.float32)


def c0_camera(n: int = 64, width: int = 128, height: int = 128) -> np.ndarray:
    """The marching workload's camera: eye (n/2, n/2, -n), looking at the centre, +y up, 40 deg."""
    c = n / 2.0
    return camera((c, c, -float(n)), (c, c, c), (0.0, 1.0, 0.0), 40.0, width, height)


# ---------------------------------------------------------------------------
# Streamline workload: v = curl A, A = sum_m a_m sin(2 pi k_m . x / n + phi_m)
# ---------------------------------------------------------------------------
def c2_modes(nmodes: int = 32, seed: int = 2, kmax: float = 8.0):
    """Integer wave vectors 1 <= |k| <= kmax, amplitudes a perpendicular to k, phases.

    Uniforms from Philox(key={seed,3}, ctr={m, j, 0, 0}); a wave vector is redrawn
    (j = 0, 2, 4, ...) until its length is in range.
    """
    ks, amps, phis = [], [], []
    for m in range(nmodes):
        j = 0
        while True:
            r = philox4x32_10(m, j, 0, 0, seed, 3)
            k = np.array([int(r[i]) % 17 - 8 for i in range(3)], np.float64)
            if 1.0 <= np.linalg.norm(k) <= kmax:
                break
            j += 2
        r2 = philox4x32_10(m, j + 1, 0, 0, seed, 3)
        u = np.array([float(r2[i]) / 4294967296.0 for i in range(4)])
        v = u[:3] * 2.0 - 1.0
        kh = k / np.linalg.norm(k)
        a = v - v.dot(kh) * kh
        if np.linalg.norm(a) < 1e-6:
            a = np.cross(kh, [1.0, 0.0, 0.0]) if abs(kh[0]) < 0.9 else np.cross(kh, [0.0, 1.0, 0.0])
        a = a / np.linalg.norm(a) * (0.5 + 0.5 * u[3])
        ks.append(k)
        amps.append(a)
        phis.append(2.0 * math.pi * (float(r[3]) / 4294967296.0))
    return np.array(ks), np.array(amps), np.array(phis)


def c2_velocity_exact(p, n: int, modes=None, scale: float = 1.0) -> np.ndarray:
    """The analytic (unscaled unless scale is given) field at points p (... x 3), float64."""
    k, a, phi = c2_modes() if modes is None else modes
    p = np.asarray(p, np.float64)
    th = 2.0 * math.pi * (p @ k.T) / n + phi          # ... x m
    w = (2.0 * math.pi / n) * np.cross(k, a)          # m x 3
    return scale * (np.cos(th) @ w)


def c2_field(n: int = 512, modes=None, zchunk: int = 16):
    """n^3 x 3 float32 velocity at voxel centres, index [z, y, x, c], scaled so max |v| = 1.

    Evaluated in float64 as a sum of separable complex exponentials (one GEMM per
    slab of z), scaled by the largest voxel speed, then rounded to float32.
    Returns (field, scale).
    """
    k, a, phi = c2_modes() if modes is None else modes
    m = len(k)
    x = (np.arange(n, dtype=np.float64) + 0.5) * (2.0 * math.pi / n)
    ex = np.exp(1j * np.outer(k[:, 0], x))            # m x n
    ey = np.exp(1j * np.outer(k[:, 1], x))
    ez = np.exp(1j * np.outer(k[:, 2], x))
    w = (2.0 * math.pi / n) * np.cross(k, a)          # m x 3
    coef = np.exp(1j * phi)                           # m

    def slab(z0, z1):
        # A[(z, y), m] = coef_m ez[m, z] ey[m, y]; v_c = Re((A * w_c) @ ex)
        zz = ez[:, z0:z1].T[:, None, :] * ey.T[None, :, :] * coef[None, None, :]   # dz x n x m
        A = zz.reshape(-1, m)
        out = np.empty((z1 - z0, n, n, 3), np.float64)
        for c in range(3):
            out[..., c] = (A * w[:, c][None, :]).dot(ex).real.reshape(z1 - z0, n, n)
        return out

    vmax = 0.0
    for z0 in range(0, n, zchunk):
        s = slab(z0, min(n, z0 + zchunk))
        vmax = max(vmax, float(np.sqrt((s * s).sum(-1)).max()))
    scale = 1.0 / vmax
    field = np.empty((n, n, n, 3), np.float32)
    for z0 in range(0, n, zchunk):
        z1 = min(n, z0 + zchunk)
        field[z0:z1] = (slab(z0, z1) * scale).astype(np.float32)
    return field, scale


def c2_seeds(count: int, n: int = 512, seed: int = 2, stream: int = 4) -> np.ndarray:
    """count x 3 float32 seed points uniform in [0, n)^3 (Philox key {seed, stream})."""
    i = np.arange(count, dtype=np.uint32)
    z = np.zeros_like(i)
    r = philox4x32_10(i, z, z, z, seed, stream)
    pts = np.stack([r[0], r[1], r[2]], 1).astype(np.float64) / 4294967296.0 * n
    return np.minimum(pts.astype(np.float32), np.float32(n) - np.float32(n) * np.float32(2**-24))


def c2_seed_set_sizes(count: int = 16) -> list:
    """Uneven batch: round(2^(12 + 8 k / 15)), k = 0 .. 15 (4096 .. 1048576)."""
    return [int(round(2 ** (12 + 8 * k / (count - 1)))) for k in range(count)]


# ---------------------------------------------------------------------------
# Differentiable rendering workload
# ---------------------------------------------------------------------------
def c3_target_volume(vol: np.ndarray, seed: int = 3, rel: float = 0.1) -> np.ndarray:
    """The target density sigma * (1 + rel * u), u uniform in [-1, 1) per voxel
    from Philox(key={seed, 6}, ctr={voxel, 0, 0, 0})."""
    i = np.arange(vol.size, dtype=np.uint32)
    z = np.zeros_like(i)
    r = philox4x32_10(i, z, z, z, seed, 6)[0]
    u = r.astype(np.float64) / 4294967296.0 * 2.0 - 1.0
    return (vol.astype(np.float64).reshape(-1) * (1.0 + rel * u)).astype(np.float32).reshape(vol.shape)


# ---------------------------------------------------------------------------
# Transport workload: fractal gradient-noise density, 4 views
# ---------------------------------------------------------------------------
_NOISE_LIB = None


def _noise_lib():
    """Build (gcc, OpenMP) and load the noise generator inputs_noise.c."""
    global _NOISE_LIB
    if _NOISE_LIB is None:
        import ctypes
        import os
        import subprocess

        here = os.path.dirname(os.path.abspath(__file__))
        src = os.path.join(here, "inputs_noise.c")
        lib = os.path.join(here, "libinputs_noise.so")
        if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            tmp = lib + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
            os.replace(tmp, lib)
        L = ctypes.CDLL(lib)
        L.noise_volume.argtypes = [ctypes.c_int32, ctypes.c_uint32, ctypes.c_int32, ctypes.c_double,
                                   ctypes.c_void_p, ctypes.c_void_p]
        L.noise_volume.restype = None
        L.noise_at.argtypes = [ctypes.c_uint32, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double]
        L.noise_at.restype = ctypes.c_double
        _NOISE_LIB = L
    return _NOISE_LIB


def noise_at(p, seed: int = 4, octaves: int = 6, base: float = 4.0) -> float:
    """Fractal gradient noise at a point of the unit cube (unclamped)."""
    return float(_noise_lib().noise_at(seed, octaves, base, float(p[0]), float(p[1]), float(p[2])))


def c4_volume(n: int = 1024, seed: int = 4, octaves: int = 6, base: float = 4.0, optical_depth: float = 8.0):
    """n^3 float32 extinction, index [z, y, x]: fractal gradient noise (octaves, base
    frequency per unit cube) clamped at 0, scaled so the mean per cell is optical_depth / n.
    Returns (volume, sigma_max)."""
    import ctypes

    vol = np.empty((n, n, n), np.float32)
    total = ctypes.c_double()
    _noise_lib().noise_volume(n, seed, octaves, base, vol.ctypes.data, ctypes.byref(total))
    mean = total.value / vol.size
    scale = np.float32((optical_depth / n) / mean)
    vol *= scale
    return vol, float(vol.max())


C4_VIEWS = ((2048, 2048), (1024, 768), (512, 512), (3840, 2160))


def c4_views(n: int = 1024, sizes=C4_VIEWS):
    """Four cameras around the grid (40 deg vertical fov, aspect of their resolution),
    as (cam float32[12], width, height, first global pixel index)."""
    c = n / 2.0
    out = []
    base = 0
    for v, (w, h) in enumerate(sizes):
        ang = math.radians(35.0 + 90.0 * v)
        eye = (c + 1.7 * n * math.sin(ang), c + 0.35 * n * (1 if v % 2 == 0 else -1), c - 1.7 * n * math.cos(ang))
        cam = camera(eye, (c, c, c), (0.0, 1.0, 0.0), 40.0, w, h)
        out.append((cam, w, h, base))
        base += w * h
    return out


# ---------------------------------------------------------------------------
# Multi-phase exchange: particles on the periodic fixed-point cube
# ---------------------------------------------------------------------------
def mp_particles(n: int, seed: int = 5, speed_bits: int = 26) -> np.ndarray:
    """``n`` 32-byte particles (n x 8 uint32: x, y, z, vx, vy, vz, m, id).

    Positions are uniform 32-bit fixed point; each velocity component is
    uniform in [-2^speed_bits, 2^speed_bits) (stored as two's complement);
    masses are 1..255; id = i.  Words from Philox(key {seed, 11}, counters
    {i, 0, 0, 0} and {i, 1, 0, 0}).
    """
    i = np.arange(n, dtype=np.uint32)
    z = np.zeros_like(i)
    a = philox4x32_10(i, z, z, z, seed, 11)
    b = philox4x32_10(i, np.ones_like(i), z, z, seed, 11)
    out = np.empty((n, 8), np.uint32)
    out[:, 0], out[:, 1], out[:, 2] = a[0], a[1], a[2]
    half = np.int64(1) << speed_bits
    for k in range(3):
        v = (b[k].astype(np.int64) >> (32 - speed_bits - 1)) - half
        out[:, 3 + k] = v.astype(np.int32).view(np.uint32)
    out[:, 6] = 1 + (a[3] >> 24) % 255
    out[:, 7] = i
    return out
