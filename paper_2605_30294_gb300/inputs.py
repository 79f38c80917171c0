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
