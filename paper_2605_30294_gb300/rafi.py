"""ctypes binding of librafi_gb.so (include/rafi.h).

Argument marshalling only: every function has the C name, takes plain ints
for device/host pointers (or objects with ``data_ptr()``, e.g. torch tensors)
and a stream handle (int, or an object with ``cuda_stream``), and raises
``RafiError`` for a status other than RF_OK unless the caller allows it.
All computation happens in the CUDA library; when the library has not been
built this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librafi_gb.so")

RF_OK, RF_ERR_ARG, RF_ERR_OOM, RF_ERR_CUDA, RF_ERR_OVERFLOW, RF_ERR_BAD_DEST, RF_ERR_MAX_ROUNDS, \
    RF_ERR_TIMEOUT, RF_ERR_STATE = range(9)
STATUS_NAMES = ["RF_OK", "RF_ERR_ARG", "RF_ERR_OOM", "RF_ERR_CUDA", "RF_ERR_OVERFLOW", "RF_ERR_BAD_DEST",
                "RF_ERR_MAX_ROUNDS", "RF_ERR_TIMEOUT", "RF_ERR_STATE"]
RF_MAX_ITEM_BYTES = 512
RF_MAX_RANKS = 1024
RF_MAX_CAPACITY = 0x7FFFFFFF
RF_C1_UNIFORM, RF_C1_ZIPF, RF_C1_NBR6 = 0, 1, 2
RF_POLICY_MICROBENCH, RF_POLICY_STREAMLINES, RF_POLICY_TRANSPORT = 0, 1, 2
RF_FORM_HOST_LOOP, RF_FORM_PERSISTENT, RF_FORM_GRAPH, RF_FORM_TUNED = 0, 1, 2, 3


class RafiError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{fn}: {name}: {msg}")


class rf_device_queues(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("dest", ctypes.c_void_p),
                ("outCount", ctypes.c_void_p), ("inOffset", ctypes.c_void_p), ("capacity", ctypes.c_uint64),
                ("itemBytes", ctypes.c_uint32), ("numRanks", ctypes.c_int32)]


class rf_round_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("numActive", "emitted", "dropped", "badDest", "holes",
                                                "exchanges", "totalDelivered", "totalDropped")]


class rf_phase_times(ctypes.Structure):
    _fields_ = [("countMs", ctypes.c_double), ("scanMs", ctypes.c_double), ("scatterMs", ctypes.c_double),
                ("workMs", ctypes.c_double), ("countLaunches", ctypes.c_uint64),
                ("scanLaunches", ctypes.c_uint64), ("scatterLaunches", ctypes.c_uint64),
                ("workLaunches", ctypes.c_uint64), ("scatterItems", ctypes.c_uint64),
                ("scatterMsLarge", ctypes.c_double), ("scatterItemsLarge", ctypes.c_uint64),
                ("scatterLaunchesLarge", ctypes.c_uint64), ("roundsMs", ctypes.c_double),
                ("roundsLaunches", ctypes.c_uint64)]


_P = ctypes.c_void_p
_i32, _u32, _u64, _f64 = ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
_PP = ctypes.POINTER(ctypes.c_void_p)
_PU64 = ctypes.POINTER(ctypes.c_uint64)

# name -> argtypes (every function returns rf_status unless listed in _RESTYPE)
_SIGS = {
    "rf_create": [_i32, _u32, _u64, _PP],
    "rf_destroy": [_P],
    "rf_resize": [_P, _u64],
    "rf_get_device_queues": [_P, ctypes.POINTER(rf_device_queues)],
    "rf_exchange": [_P, _P, _PU64],
    "rf_num_active": [_P, _PU64],
    "rf_segment": [_P, _i32, _PU64, _PU64],
    "rf_stats": [_P, ctypes.POINTER(rf_round_stats)],
    "rf_push": [_P, _P, _P, _u64, _i32, _P],
    "rf_snapshot": [_P, _P, _P, _P],
    "rf_restore": [_P, _P, _P, _u64, _P],
    "rf_set_timing": [_P, _i32],
    "rf_get_timing": [_P, ctypes.POINTER(rf_phase_times), _i32],
    "rf_set_wait_limits": [_P, _u64, _u32],
    "rf_rounds_shapes": [_i32, _P, _P, _i32],
    "rf_set_batched_config": [_P, _i32, _i32, _i32],
    "rf_get_batched_config": [_P, _i32, _P, _P],
    "rf_set_push_limit": [_P, _u64],
    "rf_get_push_limit": [_P, _P],
    "rf_set_rank_skew": [_P, _u32],
    "rf_get_rank_skew": [_P, _P],
    "rf_launch_count": [],
    "rf_last_error": [],
    "rf_partition_static": [_P, _P, _u64, _u32, _i32, _P, _P, _P, _P],
    "rf_c1_zipf_thresholds": [_i32, _f64, _P],
    "rf_c1_seed": [_P, _P, _u64, _P],
    "rf_c1_work": [_P, _u32, _u32, _i32, _f64, _i32, _i32, _i32, _P, _P, _u64, _i32, _P],
    "rf_c1_run": [_P, _P, _u64, _u32, _i32, _f64, _i32, _i32, _i32, _P, _PU64, _i32, _i32, _u32, _P,
                  _PU64, _PU64],
    "rf_c1_run_batched": [_P, _P, _u64, _u32, _i32, _f64, _i32, _i32, _i32, _P, _PU64, _i32, _i32, _u32, _P,
                          _PU64, _PU64, _P, _u32],
    "rf_c1_run_batched_runs": [_P, _P, _u64, _i32, _u32, _P, _f64, _i32, _i32, _i32, _P, _P, _i32, _u32, _P,
                               _P, _PU64, _P, _u32],
    "rf_c0_make_bricks": [_P, _i32, _i32, _P, _P],
    "rf_c2_make_bricks": [_P, _i32, _i32, _P, _P],
    "rf_c4_render": [_P, _P, _i32, _i32, ctypes.c_float, _i32, _P, _P, _i32, _u32, _P, _i32, _u32, _P, _PU64,
                     _PU64],
    "rf_c3_render": [_P, _P, _P, _i32, _i32, _i32, _i32, _i32, _u32, _P, _P, _P, _u32, _P, _PU64],
    "rf_c3_adjoint": [_P, _P, _P, _i32, _i32, _i32, _i32, _i32, _u32, _P, _P, _P, _P, _u32, _P, _PU64],
    "rf_c2_seed": [_P, _P, _P, _u64, _i32, _i32, _P],
    "rf_c2_trace": [_P, _P, _i32, _i32, ctypes.c_float, _u32, _u32, _P, _u64, _P],
    "rf_c2_run": [_P, _P, _P, _P, _u64, _i32, _i32, ctypes.c_float, _u32, _u32, _P, _i32, _u32, _P, _PU64,
                  _PU64],
    "rf_c0_raygen": [_P, _P, _i32, _i32, _i32, _i32, _P, _P],
    "rf_c0_march": [_P, _P, _i32, _i32, _P, _P, _i32, _P, _P],
    "rf_c0_render": [_P, _P, _P, _i32, _i32, _i32, _i32, _P, _P, _i32, _P, _u32, _P, _PU64],
    "rf_c0_render_graph": [_P, _P, _P, _i32, _i32, _i32, _i32, _P, _P, _i32, _P, _u32, _P, _PU64],
    "rf_c0_make_scalar_bricks": [_P, _i32, _i32, _P, _P],
    "rf_c0_march_tma": [_P, _P, _i32, _i32, _P, _P],
    "rf_c0_render_tma": [_P, _P, _P, _i32, _i32, _i32, _i32, _P, _i32, _u32, _P, _PU64],
    "rf_create_with_buffers": [_i32, _u32, _u64, _P, _P, _P, _P],
    "rf_c1_run_graph": [_P, _P, _u64, _u32, _i32, _f64, _i32, _i32, _i32, _P, _PU64, _i32, _u32, _P, _PU64, _PU64],
    "rf_get_exchange_config": [_P, _P],
    "rf_set_exchange_config": [_P, _P],
    "rf_tune_exchange": [_P, _P, _u32, _P, _P],
    "rf_mp_seed": [_P, _P, _u64, _i32, _i32, _i32, _P],
    "rf_mp_migrate": [_P, _i32, _i32, _i32, _P],
    "rf_mp_tree": [_P, _i32, _i32, _i32, _P, _P],
    "rf_mp_broadcast": [_P, _P, _P],
    "rf_mp_request": [_P, _P, _i32, _i32, _i32, _P],
    "rf_mp_respond": [_P, _P, _P, _P],
    "rf_mp_step": [_P, _P, _P, _i32, _i32, _i32, _P, _P, _PU64],
}
_RESTYPE = {"rf_launch_count": _u64, "rf_last_error": ctypes.c_char_p}

_lib = None
_lock = threading.Lock()


def lib():
    """Load librafi_gb.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with "
                                  "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = _RESTYPE.get(name, ctypes.c_int)
            _lib = L
    return _lib


def ptr(x) -> int | None:
    """Pointer value of an int, None, or an object with data_ptr() (torch tensor) / ctypes data."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):  # numpy array
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)!r}")


def stream_handle(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(fn: str, st: int, allow=()):
    if st != RF_OK and st not in allow:
        raise RafiError(st, fn, lib().rf_last_error().decode())
    return st


def rf_last_error() -> str:
    return lib().rf_last_error().decode()


def rf_set_wait_limits(ctx: int, spin_cycles: int = 0, missing_arrivals: int = 0) -> None:
    _check("rf_set_wait_limits", lib().rf_set_wait_limits(ctx, spin_cycles, missing_arrivals))


def rf_rounds_shapes(policy: int):
    """The persistent kernel's shapes for a policy: [(threads, items per thread, CTAs per SM), ...]."""
    n = ctypes.c_int32()
    _check("rf_rounds_shapes", lib().rf_rounds_shapes(policy, ctypes.byref(n), None, 0))
    arr = (ctypes.c_int32 * (3 * max(n.value, 1)))()
    _check("rf_rounds_shapes", lib().rf_rounds_shapes(policy, ctypes.byref(n), ctypes.cast(arr, _P), n.value))
    return [tuple(arr[3 * i:3 * i + 3]) for i in range(n.value)]


def rf_set_batched_config(ctx: int, policy: int, form: int, shape: int) -> None:
    _check("rf_set_batched_config", lib().rf_set_batched_config(ctx, policy, form, shape))


def rf_get_batched_config(ctx: int, policy: int):
    f, sh = ctypes.c_int32(), ctypes.c_int32()
    _check("rf_get_batched_config", lib().rf_get_batched_config(ctx, policy, ctypes.byref(f), ctypes.byref(sh)))
    return f.value, sh.value


def rf_set_push_limit(ctx: int, max_items: int) -> None:
    _check("rf_set_push_limit", lib().rf_set_push_limit(ctx, max_items))


def rf_get_push_limit(ctx: int) -> int:
    v = ctypes.c_uint64()
    _check("rf_get_push_limit", lib().rf_get_push_limit(ctx, ctypes.byref(v)))
    return v.value


def rf_set_rank_skew(ctx: int, skew: int) -> None:
    _check("rf_set_rank_skew", lib().rf_set_rank_skew(ctx, skew))


def rf_get_rank_skew(ctx: int) -> int:
    v = ctypes.c_uint32()
    _check("rf_get_rank_skew", lib().rf_get_rank_skew(ctx, ctypes.byref(v)))
    return v.value


def rf_launch_count() -> int:
    return int(lib().rf_launch_count())


def rf_create(num_ranks: int, item_bytes: int, capacity: int) -> int:
    h = ctypes.c_void_p()
    _check("rf_create", lib().rf_create(num_ranks, item_bytes, capacity, ctypes.byref(h)))
    return h.value


def rf_destroy(ctx: int) -> None:
    _check("rf_destroy", lib().rf_destroy(ctx))


def rf_resize(ctx: int, capacity: int) -> None:
    _check("rf_resize", lib().rf_resize(ctx, capacity))


def rf_get_device_queues(ctx: int) -> rf_device_queues:
    q = rf_device_queues()
    _check("rf_get_device_queues", lib().rf_get_device_queues(ctx, ctypes.byref(q)))
    return q


def rf_exchange(ctx: int, stream=None, sync: bool = True, allow=()):
    """forwardRays(): returns (status, numActive) when sync, else (status, None)."""
    n = ctypes.c_uint64()
    st = lib().rf_exchange(ctx, stream_handle(stream), ctypes.byref(n) if sync else None)
    _check("rf_exchange", st, allow)
    return st, (n.value if sync else None)


def rf_num_active(ctx: int, allow=()) -> int:
    n = ctypes.c_uint64()
    _check("rf_num_active", lib().rf_num_active(ctx, ctypes.byref(n)), allow)
    return n.value


def rf_segment(ctx: int, rank: int, allow=()):
    o, c = ctypes.c_uint64(), ctypes.c_uint64()
    _check("rf_segment", lib().rf_segment(ctx, rank, ctypes.byref(o), ctypes.byref(c)), allow)
    return o.value, c.value


def rf_stats(ctx: int, allow=()) -> rf_round_stats:
    s = rf_round_stats()
    _check("rf_stats", lib().rf_stats(ctx, ctypes.byref(s)), allow)
    return s


def rf_push(ctx: int, items, dest, n: int, host_memory: bool, stream=None) -> None:
    _check("rf_push", lib().rf_push(ctx, ptr(items), ptr(dest), n, int(host_memory), stream_handle(stream)))


def rf_snapshot(ctx: int, items_out, offsets_out, stream=None, allow=()) -> None:
    _check("rf_snapshot", lib().rf_snapshot(ctx, ptr(items_out), ptr(offsets_out), stream_handle(stream)), allow)


def rf_restore(ctx: int, items, offsets, n: int, stream=None) -> None:
    _check("rf_restore", lib().rf_restore(ctx, ptr(items), ptr(offsets), n, stream_handle(stream)))


def rf_set_timing(ctx: int, enable: bool) -> None:
    _check("rf_set_timing", lib().rf_set_timing(ctx, int(enable)))


def rf_get_timing(ctx: int, reset: bool = False, allow=()) -> rf_phase_times:
    t = rf_phase_times()
    _check("rf_get_timing", lib().rf_get_timing(ctx, ctypes.byref(t), int(reset)), allow)
    return t


def rf_partition_static(items, dest, n: int, item_bytes: int, num_ranks: int, items_out, offsets_out,
                        stats_out=None, stream=None) -> None:
    """Allocation-free stable partition into caller buffers (see rafi.h)."""
    fn = "rf_partition_static"
    _need(items, n * item_bytes, fn, "items")
    _need(items_out, n * item_bytes, fn, "items_out")
    _need(dest, n * 4, fn, "dest")
    _need(offsets_out, (max(num_ranks, 0) + 1) * 4, fn, "offsets_out")
    _need(stats_out, 32, fn, "stats_out")
    _check("rf_partition_static", lib().rf_partition_static(ptr(items), ptr(dest), n, item_bytes, num_ranks,
                                                            ptr(items_out), ptr(offsets_out), ptr(stats_out),
                                                            stream_handle(stream)))


def rf_c1_zipf_thresholds(num_ranks: int, s: float = 1.1):
    arr = (ctypes.c_uint32 * max(num_ranks, 1))()
    _check("rf_c1_zipf_thresholds", lib().rf_c1_zipf_thresholds(num_ranks, s, ctypes.cast(arr, _P)))
    return list(arr)[: max(num_ranks - 1, 0)]


def rf_c1_seed(ctx: int, items, n: int, stream=None) -> None:
    _check("rf_c1_seed", lib().rf_c1_seed(ctx, ptr(items), n, stream_handle(stream)))


def rf_c1_work(ctx: int, seed: int, hop: int, mode: int, zipf_s: float, grid, retired, retired_count,
               retired_capacity: int, deterministic: bool = False, stream=None) -> None:
    gx, gy, gz = grid
    _check("rf_c1_work", lib().rf_c1_work(ctx, seed, hop, mode, zipf_s, gx, gy, gz, ptr(retired),
                                          ptr(retired_count), retired_capacity, int(deterministic),
                                          stream_handle(stream)))


def rf_c1_run(ctx: int, items, n: int, seed: int, mode: int, zipf_s: float, grid, retired,
              deterministic: bool = False, host_memory: bool = False, max_rounds: int = 100000,
              stream=None, allow=()):
    """Whole microbenchmark; returns (status, retired_count, rounds, forwarded)."""
    gx, gy, gz = grid
    cnt, rounds, fwd = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    st = lib().rf_c1_run(ctx, ptr(items), n, seed, mode, zipf_s, gx, gy, gz, ptr(retired), ctypes.byref(cnt),
                         int(deterministic), int(host_memory), max_rounds, stream_handle(stream),
                         ctypes.byref(rounds), ctypes.byref(fwd))
    _check("rf_c1_run", st, allow)
    return st, cnt.value, rounds.value, fwd.value


def rf_c1_run_batched(ctx: int, items, n: int, seed: int, mode: int, zipf_s: float, grid, retired,
                      host_memory: bool = False, max_rounds: int = 100000, stream=None, round_log=None,
                      round_log_cap: int = 0, allow=(), step_on_arrival: bool = True):
    """Persistent-kernel microbenchmark; returns (status, retired_count, rounds, forwarded)."""
    gx, gy, gz = grid
    cnt, rounds, fwd = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    st = lib().rf_c1_run_batched(ctx, ptr(items), n, seed, mode, zipf_s, gx, gy, gz, ptr(retired),
                                 ctypes.byref(cnt), int(host_memory), int(step_on_arrival), max_rounds,
                                 stream_handle(stream),
                                 ctypes.byref(rounds), ctypes.byref(fwd), ptr(round_log), round_log_cap)
    _check("rf_c1_run_batched", st, allow)
    return st, cnt.value, rounds.value, fwd.value


def rf_c1_run_batched_runs(ctx: int, items, n: int, seed: int, modes, zipf_s: float, grid, retired,
                           host_memory: bool = False, max_rounds: int = 100000, stream=None, round_log=None,
                           round_log_cap: int = 0, allow=()):
    """Several independent microbenchmark runs (laws `modes`, n items each,
    run k at items [k n, (k + 1) n)) in one persistent launch; returns
    (status, retired counts per run, rounds per run, forwarded over all runs)."""
    fn = "rf_c1_run_batched_runs"
    k = len(modes)
    _need(items, k * n * 64, fn, "items")
    _need(retired, k * n * 64, fn, "retired")
    gx, gy, gz = grid
    m = (ctypes.c_int32 * max(k, 1))(*modes)
    cnt = (ctypes.c_uint64 * max(k, 1))()
    rounds = (ctypes.c_uint64 * max(k, 1))()
    fwd = ctypes.c_uint64()
    st = lib().rf_c1_run_batched_runs(ctx, ptr(items), n, k, seed, ctypes.cast(m, ctypes.c_void_p), zipf_s, gx, gy,
                                      gz, ptr(retired), ctypes.cast(cnt, ctypes.c_void_p), int(host_memory),
                                      max_rounds, stream_handle(stream), ctypes.cast(rounds, ctypes.c_void_p),
                                      ctypes.byref(fwd), ptr(round_log), round_log_cap)
    _check(fn, st, allow)
    return st, [int(cnt[i]) for i in range(k)], [int(rounds[i]) for i in range(k)], fwd.value


def c0_bricks_floats(n: int, brick: int) -> int:
    """Floats of the bricks rf_c0_make_bricks writes: (n/brick)^3 bricks of
    (brick+2)^3 x-y quads of 4 floats."""
    return (n // brick) ** 3 * (brick + 2) ** 3 * 4


def c0_scalar_row(brick: int) -> int:
    """Floats per row of a scalar brick: brick + 2 rounded up to a multiple of 4."""
    return (brick + 2 + 3) // 4 * 4


def c0_scalar_bricks_floats(n: int, brick: int) -> int:
    """Floats of the bricks rf_c0_make_scalar_bricks writes: (n/brick)^3 bricks of
    c0_scalar_row(brick) x (brick+2)^2 scalars."""
    return (n // brick) ** 3 * c0_scalar_row(brick) * (brick + 2) ** 2


def c2_bricks_floats(n: int, brick: int) -> int:
    """Floats of the bricks rf_c2_make_bricks writes: (n/brick)^3 bricks of
    (brick+4)^3 x-pairs of 8 floats."""
    return (n // brick) ** 3 * (brick + 4) ** 3 * 8


def _need(buf, nbytes: int, fn: str, what: str) -> None:
    """Raises RF_ERR_ARG before the call when a sized buffer (torch tensor or
    numpy array) holds fewer bytes than the call reads or writes.  Plain
    pointers (ints) cannot be checked and pass."""
    if buf is None or isinstance(buf, int):
        return
    if hasattr(buf, "numel") and hasattr(buf, "element_size"):
        have = buf.numel() * buf.element_size()
    elif hasattr(buf, "nbytes"):
        have = int(buf.nbytes)
    else:
        return
    if have < nbytes:
        raise RafiError(RF_ERR_ARG, fn, f"{what} holds {have} bytes, the call needs {nbytes}")


def _need_bricks(bricks, n: int, brick: int, fn: str, c2: bool = False) -> None:
    if brick > 0 and n > 0 and n % brick == 0:  # other shapes are refused by the library
        _need(bricks, 4 * (c2_bricks_floats(n, brick) if c2 else c0_bricks_floats(n, brick)), fn, "bricks")


def rf_c0_make_bricks(volume, n: int, brick: int, bricks, stream=None) -> None:
    _need(volume, 4 * max(n, 0) ** 3, "rf_c0_make_bricks", "volume")
    _need_bricks(bricks, n, brick, "rf_c0_make_bricks")
    _check("rf_c0_make_bricks", lib().rf_c0_make_bricks(ptr(volume), n, brick, ptr(bricks), stream_handle(stream)))


def _cam(cam):
    arr = (ctypes.c_float * 12)(*[float(x) for x in cam])
    return arr


def rf_c0_raygen(ctx: int, cam, n: int, brick: int, width: int, height: int, image, stream=None) -> None:
    c = _cam(cam)
    _check("rf_c0_raygen", lib().rf_c0_raygen(ctx, ctypes.cast(c, _P), n, brick, width, height, ptr(image),
                                              stream_handle(stream)))


def rf_c0_march(ctx: int, bricks, n: int, brick: int, image, hop_log=None, max_hops: int = 0,
                hop_count=None, stream=None) -> None:
    _need_bricks(bricks, n, brick, "rf_c0_march")
    _check("rf_c0_march", lib().rf_c0_march(ctx, ptr(bricks), n, brick, ptr(image), ptr(hop_log), max_hops,
                                            ptr(hop_count), stream_handle(stream)))


def rf_c0_render(ctx: int, bricks, cam, n: int, brick: int, width: int, height: int, image, hop_log=None,
                 max_hops: int = 0, hop_count=None, max_rounds: int = 64, stream=None) -> int:
    _need_bricks(bricks, n, brick, "rf_c0_render")
    c = _cam(cam)
    rounds = ctypes.c_uint64()
    _check("rf_c0_render", lib().rf_c0_render(ctx, ptr(bricks), ctypes.cast(c, _P), n, brick, width, height,
                                              ptr(image), ptr(hop_log), max_hops, ptr(hop_count), max_rounds,
                                              stream_handle(stream), ctypes.byref(rounds)))
    return rounds.value


def rf_c0_render_graph(ctx: int, bricks, cam, n: int, brick: int, width: int, height: int, image, hop_log=None,
                       max_hops: int = 0, hop_count=None, max_rounds: int = 64, stream=None) -> int:
    """rf_c0_render with the rounds in a kept CUDA graph (conditional while node)."""
    _need_bricks(bricks, n, brick, "rf_c0_render_graph")
    c = _cam(cam)
    rounds = ctypes.c_uint64()
    _check("rf_c0_render_graph", lib().rf_c0_render_graph(ctx, ptr(bricks), ctypes.cast(c, _P), n, brick, width,
                                                          height, ptr(image), ptr(hop_log), max_hops,
                                                          ptr(hop_count), max_rounds, stream_handle(stream),
                                                          ctypes.byref(rounds)))
    return rounds.value


RF_C2_EXITED, RF_C2_STALLED, RF_C2_MAXSTEPS = 1, 2, 3


def rf_c2_make_bricks(field, n: int, brick: int, bricks, stream=None) -> None:
    _need(field, 12 * max(n, 0) ** 3, "rf_c2_make_bricks", "field")
    _need_bricks(bricks, n, brick, "rf_c2_make_bricks", c2=True)
    _check("rf_c2_make_bricks", lib().rf_c2_make_bricks(ptr(field), n, brick, ptr(bricks), stream_handle(stream)))


def rf_c2_seed(ctx: int, seeds, set_ids, count: int, n: int, brick: int, stream=None) -> None:
    _check("rf_c2_seed", lib().rf_c2_seed(ctx, ptr(seeds), ptr(set_ids), count, n, brick, stream_handle(stream)))


def rf_c2_trace(ctx: int, bricks, n: int, brick: int, h: float, max_steps: int, steps_per_round: int, out,
                out_capacity: int, stream=None) -> None:
    _need_bricks(bricks, n, brick, "rf_c2_trace", c2=True)
    _check("rf_c2_trace", lib().rf_c2_trace(ctx, ptr(bricks), n, brick, h, max_steps, steps_per_round, ptr(out),
                                            out_capacity, stream_handle(stream)))


def rf_c2_run(ctx: int, bricks, seeds, set_ids, count: int, n: int, brick: int, h: float, max_steps: int,
              steps_per_round: int, out, batched: bool, max_rounds: int = 1 << 20, stream=None, allow=()):
    """Whole streamline run; returns (status, rounds, forwarded)."""
    _need_bricks(bricks, n, brick, "rf_c2_run", c2=True)
    rounds, fwd = ctypes.c_uint64(), ctypes.c_uint64()
    st = lib().rf_c2_run(ctx, ptr(bricks), ptr(seeds), ptr(set_ids), count, n, brick, h, max_steps,
                         steps_per_round, ptr(out), int(batched), max_rounds, stream_handle(stream),
                         ctypes.byref(rounds), ctypes.byref(fwd))
    _check("rf_c2_run", st, allow)
    return st, rounds.value, fwd.value


def rf_c3_render(ctx: int, bricks, cam, n: int, brick: int, width: int, height: int, spp: int, seed: int, ray_c,
                 image, max_rounds: int = 64, stream=None, ray_c_lo=None) -> int:
    _need_bricks(bricks, n, brick, "rf_c3_render")
    nr = max(width, 0) * max(height, 0) * max(spp, 0)
    _need(ray_c, 4 * nr, "rf_c3_render", "ray_c")
    _need(ray_c_lo, 4 * nr, "rf_c3_render", "ray_c_lo")
    _need(image, 4 * max(width, 0) * max(height, 0), "rf_c3_render", "image")
    c = _cam(cam)
    rounds = ctypes.c_uint64()
    _check("rf_c3_render", lib().rf_c3_render(ctx, ptr(bricks), ctypes.cast(c, _P), n, brick, width, height, spp,
                                              seed, ptr(ray_c), ptr(ray_c_lo), ptr(image), max_rounds,
                                              stream_handle(stream), ctypes.byref(rounds)))
    return rounds.value


def rf_c3_adjoint(ctx: int, bricks, cam, n: int, brick: int, width: int, height: int, spp: int, seed: int, ray_c,
                  grad_image, grad_volume, max_rounds: int = 64, stream=None, ray_c_lo=None) -> int:
    _need_bricks(bricks, n, brick, "rf_c3_adjoint")
    nr = max(width, 0) * max(height, 0) * max(spp, 0)
    _need(ray_c, 4 * nr, "rf_c3_adjoint", "ray_c")
    _need(ray_c_lo, 4 * nr, "rf_c3_adjoint", "ray_c_lo")
    _need(grad_image, 4 * max(width, 0) * max(height, 0), "rf_c3_adjoint", "grad_image")
    _need(grad_volume, 4 * max(n, 0) ** 3, "rf_c3_adjoint", "grad_volume")
    c = _cam(cam)
    rounds = ctypes.c_uint64()
    _check("rf_c3_adjoint", lib().rf_c3_adjoint(ctx, ptr(bricks), ctypes.cast(c, _P), n, brick, width, height, spp,
                                                seed, ptr(ray_c), ptr(ray_c_lo), ptr(grad_image), ptr(grad_volume),
                                                max_rounds, stream_handle(stream), ctypes.byref(rounds)))
    return rounds.value


def rf_c4_render(ctx: int, bricks, n: int, brick: int, sigma_max: float, views, spp: int, seed: int, score,
                 batched: bool = True, max_rounds: int = 1 << 20, stream=None):
    """views: sequence of (cam[12], width, height, ...); returns (rounds, forwarded)."""
    _need_bricks(bricks, n, brick, "rf_c4_render")
    nv = len(views)
    cams = (ctypes.c_float * (12 * nv))(*[float(x) for v in views for x in v[0]])
    sizes = (ctypes.c_int32 * (2 * nv))(*[int(x) for v in views for x in (v[1], v[2])])
    rounds, fwd = ctypes.c_uint64(), ctypes.c_uint64()
    _check("rf_c4_render", lib().rf_c4_render(ctx, ptr(bricks), n, brick, sigma_max, nv, ctypes.cast(cams, _P),
                                              ctypes.cast(sizes, _P), spp, seed, ptr(score), int(batched),
                                              max_rounds, stream_handle(stream), ctypes.byref(rounds),
                                              ctypes.byref(fwd)))
    return rounds.value, fwd.value


class Context:
    """Owning handle of an rf_ctx (host context of Sec. 3.4)."""

    def __init__(self, num_ranks: int, item_bytes: int, capacity: int, buffers=None):
        """buffers: optional (in_queue, out_queue, dest) device buffers the caller owns."""
        if buffers is None:
            self.handle = rf_create(num_ranks, item_bytes, capacity)
        else:
            self.handle = rf_create_with_buffers(num_ranks, item_bytes, capacity, *buffers)
        self.buffers = buffers  # keeps caller-owned queues alive while the context uses them
        self.num_ranks, self.item_bytes, self.capacity = num_ranks, item_bytes, capacity

    def close(self):
        if self.handle:
            rf_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- multi-phase exchange (three contexts) ---------------------------------
def rf_mp_seed(ctx: int, particles, n: int, grid, stream=None) -> None:
    _check("rf_mp_seed", lib().rf_mp_seed(ctx, ptr(particles), n, *grid, stream_handle(stream)))


def rf_mp_migrate(ctx: int, grid, stream=None) -> None:
    _check("rf_mp_migrate", lib().rf_mp_migrate(ctx, *grid, stream_handle(stream)))


def rf_mp_tree(ctx: int, grid, nodes, stream=None) -> None:
    _check("rf_mp_tree", lib().rf_mp_tree(ctx, *grid, ptr(nodes), stream_handle(stream)))


def rf_mp_broadcast(node_ctx: int, nodes, stream=None) -> None:
    _check("rf_mp_broadcast", lib().rf_mp_broadcast(node_ctx, ptr(nodes), stream_handle(stream)))


def rf_mp_request(node_ctx: int, request_ctx: int, grid, stream=None) -> None:
    _check("rf_mp_request", lib().rf_mp_request(node_ctx, request_ctx, *grid, stream_handle(stream)))


def rf_mp_respond(request_ctx: int, node_ctx: int, nodes, stream=None) -> None:
    _check("rf_mp_respond", lib().rf_mp_respond(request_ctx, node_ctx, ptr(nodes), stream_handle(stream)))


def rf_mp_step(particle_ctx: int, node_ctx: int, request_ctx: int, grid, nodes, stream=None):
    """One protocol step; returns the items delivered by its four exchanges."""
    got = (ctypes.c_uint64 * 4)()
    _check("rf_mp_step", lib().rf_mp_step(particle_ctx, node_ctx, request_ctx, *grid, ptr(nodes),
                                          stream_handle(stream), got))
    return tuple(int(v) for v in got)


# --- exchange configuration and autotuner ----------------------------------
class ExchangeConfig(ctypes.Structure):
    _fields_ = [("tileItems", ctypes.c_uint32), ("scatterBlocks", ctypes.c_int32), ("countBlocks", ctypes.c_int32)]

    def as_tuple(self):
        return (int(self.tileItems), int(self.scatterBlocks), int(self.countBlocks))


def rf_get_exchange_config(ctx: int):
    """(tileItems, scatterBlocks, countBlocks) of the context's exchange."""
    cfg = ExchangeConfig()
    _check("rf_get_exchange_config", lib().rf_get_exchange_config(ctx, ctypes.byref(cfg)))
    return cfg.as_tuple()


def rf_set_exchange_config(ctx: int, tile_items: int = 0, scatter_blocks: int = 0, count_blocks: int = 0,
                           allow=()) -> int:
    cfg = ExchangeConfig(tile_items, scatter_blocks, count_blocks)
    st = lib().rf_set_exchange_config(ctx, ctypes.byref(cfg))
    _check("rf_set_exchange_config", st, allow)
    return st


def rf_tune_exchange(ctx: int, stream=None, trials: int = 3):
    """Tune on the current out-queue; returns ((tileItems, scatterBlocks, countBlocks), ms)."""
    cfg = ExchangeConfig()
    ms = ctypes.c_float()
    _check("rf_tune_exchange", lib().rf_tune_exchange(ctx, stream_handle(stream), trials, ctypes.byref(cfg),
                                                      ctypes.byref(ms)))
    return cfg.as_tuple(), float(ms.value)


def rf_create_with_buffers(num_ranks: int, item_bytes: int, capacity: int, in_queue, out_queue, dest) -> int:
    """A context over caller-owned device queues; returns its handle (close it with rf_destroy)."""
    h = ctypes.c_void_p()
    _check("rf_create_with_buffers", lib().rf_create_with_buffers(num_ranks, item_bytes, capacity, ptr(in_queue),
                                                                  ptr(out_queue), ptr(dest), ctypes.byref(h)))
    return h.value


def rf_c1_run_graph(ctx: int, items, n: int, seed: int, mode: int, zipf_s: float, grid, retired,
                    deterministic: bool = True, max_rounds: int = 100000, stream=None, allow=()):
    """Microbenchmark with the rounds in a CUDA graph; returns (status, retired_count, rounds, forwarded)."""
    gx, gy, gz = grid
    cnt, rounds, fwd = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    st = lib().rf_c1_run_graph(ctx, ptr(items), n, seed, mode, zipf_s, gx, gy, gz, ptr(retired), ctypes.byref(cnt),
                               int(deterministic), max_rounds, stream_handle(stream), ctypes.byref(rounds),
                               ctypes.byref(fwd))
    _check("rf_c1_run_graph", st, allow)
    return st, cnt.value, rounds.value, fwd.value


def rf_c0_make_scalar_bricks(volume, n: int, brick: int, bricks, stream=None) -> None:
    _need(volume, 4 * max(n, 0) ** 3, "rf_c0_make_scalar_bricks", "volume")
    if brick > 0 and n > 0 and n % brick == 0:
        _need(bricks, 4 * c0_scalar_bricks_floats(n, brick), "rf_c0_make_scalar_bricks", "bricks")
    _check("rf_c0_make_scalar_bricks", lib().rf_c0_make_scalar_bricks(ptr(volume), n, brick, ptr(bricks),
                                                                      stream_handle(stream)))


def rf_c0_render_tma(ctx: int, scalar_bricks, cam, n: int, brick: int, width: int, height: int, image,
                     max_rounds: int = 16, stream=None, form: int = RF_FORM_HOST_LOOP) -> int:
    """Marching with each brick staged in shared memory by a tensor copy, as the host
    loop or the graph loop (form); returns rounds."""
    if brick > 0 and n > 0 and n % brick == 0:
        _need(scalar_bricks, 4 * c0_scalar_bricks_floats(n, brick), "rf_c0_render_tma", "scalar_bricks")
    _need(image, 4 * max(width, 0) * max(height, 0), "rf_c0_render_tma", "image")
    c = _cam(cam)
    rounds = ctypes.c_uint64()
    _check("rf_c0_render_tma", lib().rf_c0_render_tma(ctx, ptr(scalar_bricks), ctypes.cast(c, _P), n, brick, width,
                                                      height, ptr(image), form, max_rounds, stream_handle(stream),
                                                      ctypes.byref(rounds)))
    return rounds.value


def rf_c0_march_tma(ctx: int, scalar_bricks, n: int, brick: int, image, stream=None) -> None:
    """One marching round with TMA-staged bricks over the context's incoming queue."""
    if brick > 0 and n > 0 and n % brick == 0:
        _need(scalar_bricks, 4 * c0_scalar_bricks_floats(n, brick), "rf_c0_march_tma", "scalar_bricks")
    _check("rf_c0_march_tma", lib().rf_c0_march_tma(ctx, ptr(scalar_bricks), n, brick, ptr(image),
                                                    stream_handle(stream)))
