"""Oracle for the RaFI work-forwarding hot path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never does: it shares no code with the oracle.

The arithmetic lives in ``oracle.c`` (plain single-threaded C, built without
FMA contraction); this module only builds it and marshals numpy arrays.
Every function cites the passage of the paper it restates.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

UNIFORM, ZIPF, NBR6 = 0, 1, 2
RETIRE_THRESHOLD = 429496730  # ceil(0.1 * 2**32)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, no FMA contraction)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            u32, i32, u64, f64 = ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
            lib.or_philox_batch.argtypes = [u64, P, P, P]
            lib.or_philox_batch.restype = None
            lib.or_partition.argtypes = [P, P, u64, u32, i32, P, P, P, P]
            lib.or_partition.restype = u64
            lib.or_zipf_thresholds.argtypes = [i32, f64, P]
            lib.or_zipf_thresholds.restype = None
            lib.or_c1_choose_dest.argtypes = [i32, i32, u32, i32, P, P]
            lib.or_c1_choose_dest.restype = i32
            lib.or_c1_walk.argtypes = [P, u64, i32, u32, i32, P, P, u32, P, P, P, P]
            lib.or_c1_walk.restype = u64
            lib.or_c1_rounds.argtypes = [P, u64, i32, u32, i32, P, P, u32, P, P, P, i32, P, P]
            lib.or_c1_rounds.restype = i32
            lib.or_c0_primary.argtypes = [P, i32, i32, i32, P, P, P]
            lib.or_c0_primary.restype = i32
            lib.or_c0_render.argtypes = [P, i32, i32, P, i32, i32, P, P, P, P, i32, P]
            lib.or_c0_render.restype = None
            lib.or_c0_sigma.argtypes = [P, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float]
            lib.or_c0_sigma.restype = ctypes.c_float
            lib.or_c2_rk4.argtypes = [P, i32, ctypes.c_float, P, P]
            lib.or_c2_rk4.restype = None
            lib.or_c2_velocity.argtypes = [P, i32, P, P]
            lib.or_c2_velocity.restype = None
            lib.or_c2_trace.argtypes = [P, i32, i32, P, u64, ctypes.c_float, u32, P, P, P, P]
            lib.or_c2_trace.restype = None
            lib.or_c3_render.argtypes = [P, i32, P, i32, i32, i32, u32, P, P]
            lib.or_c3_render.restype = None
            lib.or_c3_adjoint_f64.argtypes = [P, i32, P, i32, i32, i32, u32, P, P, P, P]
            lib.or_c3_adjoint_f64.restype = f64
            lib.or_c4_path.argtypes = [P, i32, ctypes.c_float, P, i32, i32, i32, u32, u32, u32, P, P]
            lib.or_c4_path.restype = i32
            lib.or_c4_render_crop.argtypes = [P, i32, ctypes.c_float, P, i32, u32, i32, i32, i32, i32, i32, u32,
                                              P, P]
            lib.or_c4_render_crop.restype = None
            lib.or_c4_hg_sample.argtypes = [P, ctypes.c_float, ctypes.c_float, P]
            lib.or_c4_hg_sample.restype = None
            lib.or_mp_owner.argtypes = [u32, u32, u32, P]
            lib.or_mp_owner.restype = i32
            lib.or_mp_migrate.argtypes = [P, u64, P, P, P]
            lib.or_mp_migrate.restype = None
            lib.or_mp_tree.argtypes = [P, u64, P, P]
            lib.or_mp_tree.restype = None
            lib.or_mp_near.argtypes = [i32, i32, P]
            lib.or_mp_near.restype = i32
            _lib = lib
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11)
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of counters ``ctr`` (n x 4 uint32) under keys ``key`` (n x 2)."""
    ctr = _c(np.atleast_2d(ctr), np.uint32)
    key = _c(np.broadcast_to(np.atleast_2d(key), (ctr.shape[0], 2)), np.uint32)
    out = np.empty_like(ctr)
    _load().or_philox_batch(ctr.shape[0], _p(ctr), _p(key), _p(out))
    return out


# --------------------------------------------------------------------------
# Exchange: stable partition by destination (Sec. 4.2.1-4.2.3)
# --------------------------------------------------------------------------
def partition(items: np.ndarray, dest: np.ndarray, num_ranks: int):
    """Stable partition of ``items`` (n x itemBytes uint8) by ``dest``.

    Returns (out, offset[R+1], bad, holes): ``out[offset[r]:offset[r+1]]`` is
    rank r's next incoming queue, in emission order (Sec. 4.2.1's radix sort
    on (dest << 32 | i) followed by the gather).
    """
    items = _c(items, np.uint8)
    dest = _c(dest, np.int32)
    n = dest.shape[0]
    item_bytes = items.shape[1] if n else (items.shape[1] if items.ndim == 2 else 0)
    out = np.zeros((n, item_bytes), np.uint8)
    off = np.zeros(num_ranks + 1, np.uint64)
    bad = np.zeros(1, np.uint64)
    holes = np.zeros(1, np.uint64)
    total = _load().or_partition(_p(items), _p(dest), n, item_bytes, num_ranks, _p(out), _p(off),
                                 _p(bad), _p(holes))
    return out[:total], off, int(bad[0]), int(holes[0])


# --------------------------------------------------------------------------
# Forwarding microbenchmark
# --------------------------------------------------------------------------
def zipf_thresholds(num_ranks: int, s: float = 1.1) -> np.ndarray:
    thr = np.zeros(max(num_ranks - 1, 1), np.uint32)
    _load().or_zipf_thresholds(num_ranks, s, _p(thr))
    return thr[: max(num_ranks - 1, 0)]


def _grid_of(num_ranks: int, grid):
    if grid is None:
        return np.array([num_ranks, 1, 1], np.int32)
    return _c(grid, np.int32)


def choose_dest(mode: int, src: int, r1: int, num_ranks: int, grid=None, thr=None) -> int:
    g = _grid_of(num_ranks, grid)
    t = zipf_thresholds(num_ranks) if thr is None else _c(thr, np.uint32)
    t = t if t.size else np.zeros(1, np.uint32)
    return int(_load().or_c1_choose_dest(mode, src, r1, num_ranks, _p(g), _p(t)))


def c1_walk(items: np.ndarray, num_ranks: int, seed: int, mode: int, grid=None, thr=None,
            max_hops: int = 100000, record_visits: bool = False, start_ranks=None):
    """Walk each item until it retires (item i starts on start_ranks[i], default i mod R).

    Returns (final n x 16, hops n, unfinished, visits).
    """
    items = _c(items, np.uint32).reshape(-1, 16)
    n = items.shape[0]
    sr = None if start_ranks is None else _c(start_ranks, np.int32)
    g = _grid_of(num_ranks, grid)
    t = zipf_thresholds(num_ranks) if thr is None else _c(thr, np.uint32)
    t = t if t.size else np.zeros(1, np.uint32)
    final = np.empty_like(items)
    hops = np.empty(n, np.uint32)
    visits = np.full((n, max_hops), -1, np.int32) if record_visits else None
    unfinished = _load().or_c1_walk(_p(items), n, num_ranks, seed, mode, _p(g), _p(t), max_hops, _p(sr),
                                    _p(final), _p(hops), _p(visits))
    return final, hops, int(unfinished), visits


def c1_rounds(items: np.ndarray, num_ranks: int, seed: int, mode: int, grid=None, thr=None,
              max_rounds: int = 100000, dump_round: int = -1):
    """Round-by-round queue simulation.

    Returns dict(rounds, active[rounds+1], retired[rounds], retired_items,
    dump_items, dump_offsets).
    """
    items = _c(items, np.uint32).reshape(-1, 16)
    n = items.shape[0]
    g = _grid_of(num_ranks, grid)
    t = zipf_thresholds(num_ranks) if thr is None else _c(thr, np.uint32)
    t = t if t.size else np.zeros(1, np.uint32)
    active = np.zeros(max_rounds + 2, np.uint64)
    retired = np.zeros(max_rounds + 2, np.uint64)
    retired_items = np.zeros((max(n, 1), 16), np.uint32)
    dump_items = np.zeros((max(n, 1), 16), np.uint32) if dump_round >= 0 else None
    dump_off = np.zeros(num_ranks + 1, np.uint64) if dump_round >= 0 else None
    rounds = _load().or_c1_rounds(_p(items), n, num_ranks, seed, mode, _p(g), _p(t), max_rounds,
                                  _p(active), _p(retired), _p(retired_items), dump_round,
                                  _p(dump_items), _p(dump_off))
    if rounds < 0:
        raise RuntimeError("oracle: max_rounds reached")
    res = dict(rounds=rounds, active=active[: rounds + 1].copy(), retired=retired[:rounds].copy(),
               retired_items=retired_items[:n])
    if dump_round >= 0:
        cnt = int(dump_off[-1]) if dump_round <= rounds else 0
        res["dump_items"] = dump_items[:cnt]
        res["dump_offsets"] = dump_off
    return res


# --------------------------------------------------------------------------
# Absorption marching (Sec. 5.1 trace step, absorption only)
# --------------------------------------------------------------------------
def c0_primary(cam: np.ndarray, n: int, x: int, y: int):
    cam = _c(cam, np.float32)
    d = np.zeros(3, np.float32)
    t0 = np.zeros(1, np.float32)
    t1 = np.zeros(1, np.float32)
    hit = _load().or_c0_primary(_p(cam), n, x, y, _p(d), _p(t0), _p(t1))
    return bool(hit), d, float(t0[0]), float(t1[0])


def c0_render(vol: np.ndarray, cam: np.ndarray, width: int, height: int, brick: int | None = None,
              max_hops: int = 16):
    """Render through the unpartitioned volume.  Returns dict(T, tau, nsamp, hops, hop_count)."""
    vol = _c(vol, np.float32)
    n = vol.shape[0]
    b = n if brick is None else brick
    cam = _c(cam, np.float32)
    npx = width * height
    T = np.zeros(npx, np.float32)
    tau = np.zeros(npx, np.float32)
    ns = np.zeros(npx, np.int32)
    hop = np.full((npx, max_hops), -1, np.int32)
    hc = np.zeros(npx, np.int32)
    _load().or_c0_render(_p(vol), n, b, _p(cam), width, height, _p(T), _p(tau), _p(ns), _p(hop),
                         max_hops, _p(hc))
    return dict(T=T, tau=tau, nsamp=ns, hops=hop, hop_count=hc)


def c0_sigma(vol: np.ndarray, p) -> float:
    vol = _c(vol, np.float32)
    return float(_load().or_c0_sigma(_p(vol), vol.shape[0], float(p[0]), float(p[1]), float(p[2])))


# --------------------------------------------------------------------------
# Streamlines (Sec. 5.4): RK4 through a trilinear vector field
# --------------------------------------------------------------------------
EXITED, STALLED, MAXSTEPS = 1, 2, 3


def c2_velocity(field: np.ndarray, p) -> np.ndarray:
    field = _c(field, np.float32)
    q = _c(np.asarray(p, np.float32).reshape(3), np.float32)
    out = np.zeros(3, np.float32)
    _load().or_c2_velocity(_p(field), field.shape[0], _p(q), _p(out))
    return out


def c2_rk4(field: np.ndarray, p, h: float = 0.25) -> np.ndarray:
    field = _c(field, np.float32)
    q = _c(np.asarray(p, np.float32).reshape(3), np.float32)
    out = np.zeros(3, np.float32)
    _load().or_c2_rk4(_p(field), field.shape[0], h, _p(q), _p(out))
    return out


def c2_trace(field: np.ndarray, seeds: np.ndarray, brick: int, h: float = 0.25, max_steps: int = 2000):
    """Trace particles through the unpartitioned field (field: N x N x N x 3, index [z, y, x, c]).

    Returns dict(pos n x 3, steps, hops, status).
    """
    field = _c(field, np.float32)
    seeds = _c(seeds, np.float32).reshape(-1, 3)
    n = seeds.shape[0]
    pos = np.zeros((n, 3), np.float32)
    steps = np.zeros(n, np.uint32)
    hops = np.zeros(n, np.uint32)
    status = np.zeros(n, np.uint32)
    _load().or_c2_trace(_p(field), field.shape[0], brick, _p(seeds), n, h, max_steps, _p(pos), _p(steps),
                        _p(hops), _p(status))
    return dict(pos=pos, steps=steps, hops=hops, status=status)


# --------------------------------------------------------------------------
# Differentiable emission-absorption rendering (Sec. 5.2's integration model)
# --------------------------------------------------------------------------
def c3_render(vol: np.ndarray, cam: np.ndarray, width: int, height: int, spp: int, seed: int = 3):
    """Float forward render: returns (image W*H, per-sample C W*H*spp)."""
    vol = _c(vol, np.float32)
    cam = _c(cam, np.float32)
    rayC = np.zeros(width * height * spp, np.float32)
    image = np.zeros(width * height, np.float32)
    _load().or_c3_render(_p(vol), vol.shape[0], _p(cam), width, height, spp, seed, _p(rayC), _p(image))
    return image, rayC


def c3_adjoint_f64(vol: np.ndarray, cam: np.ndarray, width: int, height: int, spp: int, dLdC: np.ndarray,
                   seed: int = 3, with_abs: bool = False):
    """Reference gradient dL/dvol (float64, N^3) for per-sample dL/dC (W*H*spp)
    (Sec. 5.2 integration, adjoint by reverse accumulation).  Returns (grad, acc),
    or (grad, acc, gabs, count) with gabs the per-voxel sum, over the contributions,
    of |dL/dC| x (|first part| + |0.5 S|) x weight (the rounding scale) and count
    the number of (sample, corner) contributions per voxel."""
    vol = _c(vol, np.float32)
    cam = _c(cam, np.float32)
    g = _c(dLdC, np.float64)
    grad = np.zeros(vol.shape, np.float64)
    gabs = np.zeros(vol.shape, np.float64) if with_abs else None
    cnt = np.zeros(vol.shape, np.float64) if with_abs else None
    acc = _load().or_c3_adjoint_f64(_p(vol), vol.shape[0], _p(cam), width, height, spp, seed, _p(g), _p(grad),
                                    _p(gabs), _p(cnt))
    return (grad, acc, gabs, cnt) if with_abs else (grad, acc)


# --------------------------------------------------------------------------
# Delta-tracking transport (Sec. 5.1's trace step with scattering)
# --------------------------------------------------------------------------
def c4_path(vol, sigma_max, cam, width, x, y, gpix, s, seed=4):
    """Score, events and bounces of one path."""
    vol = _c(vol, np.float32)
    cam = _c(cam, np.float32)
    ev = np.zeros(1, np.uint32)
    bo = np.zeros(1, np.uint32)
    sc = _load().or_c4_path(_p(vol), vol.shape[0], sigma_max, _p(cam), width, x, y, gpix, s, seed, _p(ev), _p(bo))
    return int(sc), int(ev[0]), int(bo[0])


def c4_render_crop(vol, sigma_max, cam, width, pix_base, x0, y0, cw, ch, spp, seed=4):
    """Mean path score over spp per pixel of a crop (ch x cw) and the number of events."""
    vol = _c(vol, np.float32)
    cam = _c(cam, np.float32)
    img = np.zeros(cw * ch, np.float32)
    ev = np.zeros(1, np.uint64)
    _load().or_c4_render_crop(_p(vol), vol.shape[0], sigma_max, _p(cam), width, pix_base, x0, y0, cw, ch, spp,
                              seed, _p(img), _p(ev))
    return img.reshape(ch, cw), int(ev[0])


def c4_hg_sample(d, xi: float, xphi: float) -> np.ndarray:
    d = _c(np.asarray(d, np.float32).reshape(3), np.float32)
    out = np.zeros(3, np.float32)
    _load().or_c4_hg_sample(_p(d), xi, xphi, _p(out))
    return out


# --------------------------------------------------------------------------
# Multi-phase exchange with three item types (Sec. 5.5's protocol:
# migration, root broadcast, refinement requests, child replies)
# --------------------------------------------------------------------------
MP_ROOT_CODE = 0  # node code of a root; child octant o has code 1 + o


def _lg(grid):
    lg = [int(g).bit_length() - 1 for g in grid]
    assert all(1 << l == g for l, g in zip(lg, grid)), "grid sides must be powers of two"
    return np.array(lg, dtype=np.int32)


def mp_owner(x: int, y: int, z: int, grid) -> int:
    """Rank owning fixed-point position (x, y, z) on a grid of ranks."""
    return int(_load().or_mp_owner(x, y, z, _p(_lg(grid))))


def mp_migrate(particles: np.ndarray, grid):
    """Move every particle (n x 8 uint32) by its velocity; returns (moved, owner)."""
    p = _c(particles, np.uint32).reshape(-1, 8)
    out = np.zeros_like(p)
    owner = np.zeros(len(p), np.int32)
    _load().or_mp_migrate(_p(p), len(p), _p(_lg(grid)), _p(out), _p(owner))
    return out, owner


def mp_tree(particles: np.ndarray, grid) -> np.ndarray:
    """Per-rank nodes (R x 9 x 5 uint64: M, X, Y, Z, count; root then octants)."""
    p = _c(particles, np.uint32).reshape(-1, 8)
    lg = _lg(grid)
    nodes = np.zeros((1 << int(lg.sum()), 9, 5), np.uint64)
    _load().or_mp_tree(_p(p), len(p), _p(lg), _p(nodes))
    return nodes


def mp_near(r: int, s: int, grid) -> bool:
    return bool(_load().or_mp_near(r, s, _p(_lg(grid))))


def mp_node_item(nd, src: int, code: int) -> np.ndarray:
    """The 64-byte node item: M, X, Y, Z as uint64 words, count, source rank, code, level."""
    w = np.zeros(16, np.uint32)
    w[0:8] = np.asarray(nd[:4], np.uint64).view(np.uint32)
    w[8], w[9], w[10], w[11] = int(nd[4]), src, code, 0 if code == MP_ROOT_CODE else 1
    return w


def mp_protocol(particles: np.ndarray, grid):
    """One step of the protocol, per rank: the migrated particles it owns, the
    roots it receives (every other rank's), the requests it receives (from
    near peers whose copy of its root is non-empty) and the children it
    receives (the non-empty octants of every near peer it asked)."""
    moved, owner = mp_migrate(particles, grid)
    R = int(np.prod(grid))
    nodes = mp_tree(moved, grid)
    near = np.array([[mp_near(r, s, grid) for s in range(R)] for r in range(R)])
    out = {"moved": moved, "owner": owner, "nodes": nodes,
           "particles_at": [moved[owner == r] for r in range(R)], "roots_at": [], "requests_at": [],
           "children_at": []}
    for r in range(R):
        out["roots_at"].append(np.array([mp_node_item(nodes[s, 0], s, MP_ROOT_CODE) for s in range(R) if s != r],
                                        np.uint32).reshape(-1, 16))
    asks = [[s for s in range(R) if near[r, s] and nodes[s, 0, 4] > 0] for r in range(R)]
    for s in range(R):
        out["requests_at"].append(np.array([[r, s, MP_ROOT_CODE, 0] for r in range(R) if s in asks[r]],
                                           np.uint32).reshape(-1, 4))
    for r in range(R):
        out["children_at"].append(np.array([mp_node_item(nodes[s, 1 + o], s, 1 + o) for s in asks[r]
                                            for o in range(8) if nodes[s, 1 + o, 4] > 0],
                                           np.uint32).reshape(-1, 16))
    return out
