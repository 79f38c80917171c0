"""Autotuner of the batched form.

For one workload policy (RF_POLICY_MICROBENCH, _STREAMLINES or _TRANSPORT) it
times every candidate configuration on a sample of the caller's run and
leaves the fastest set on the context (rf_set_batched_config):

  * the form of a run: the per-round host loop, all rounds in one persistent
    cooperative kernel, or the round's kernels in a CUDA graph whose
    conditional while node repeats them (the microbenchmark's batched call is
    always persistent);
  * the persistent kernel's shape: threads per CTA, items per thread per
    tile (the scatter's bucket tile) and resident CTAs per SM, one compiled
    variant each (rf_rounds_shapes).

Queue capacity is not a candidate: it is the caller's bound on items in
flight (rf_create / rf_resize, the paper's resizeRayQueues), and a smaller one
would drop items instead of running faster.

The winner is cached in a JSON file keyed by GPU name, policy, item size,
rank count, the sample's size (as a power-of-two bucket) and a caller-given
tag (for example the steps per round), so that later runs on the same kind
of GPU skip the timing.  This module is host-side orchestration only: every
candidate runs through the library's own calls, and the choice changes
timings, never results (every shape computes the same rounds bit for bit).
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import rafi

_lock = threading.Lock()


def cache_path() -> str:
    """RAFI_TUNE_CACHE, else ~/.cache/rafi_gb300/tune.json."""
    return os.environ.get("RAFI_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "rafi_gb300",
                                                            "tune.json")


def cache_key(gpu: str, policy: int, item_bytes: int, ranks: int, n: int, tag: str = "") -> str:
    bucket = int(math.log2(n)) if n > 0 else 0
    return f"{gpu}|policy={policy}|item_bytes={item_bytes}|ranks={ranks}|n=2^{bucket}|{tag}"


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, key: str, value: dict) -> None:
    with _lock:
        data = _load(path)
        data[key] = value
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def candidates(policy: int, forms) -> list[tuple[int, int]]:
    """(form, shape) pairs: every compiled shape for the persistent form, shape 0 otherwise."""
    nshapes = len(rafi.rf_rounds_shapes(policy))
    out = []
    for form in forms:
        out += [(form, s) for s in range(nshapes)] if form == rafi.RF_FORM_PERSISTENT else [(form, 0)]
    return out


def tune(ctx: int, policy: int, run, *, item_bytes: int, ranks: int, n: int, tag: str = "",
         forms=(rafi.RF_FORM_PERSISTENT,), reps: int = 2, use_cache: bool = True, path: str | None = None,
         stream=None) -> dict:
    """Times run() once per repetition for each candidate and keeps the fastest.

    run(form) must perform one run of the sample through the library with the
    context as configured (for rf_c2_run / rf_c4_render: batched=RF_FORM_TUNED,
    or `form` itself).  Returns {"form", "shape", "threads", "items_per_thread",
    "ctas_per_sm", "ms", "cached", "candidates": [...]}; the context is left set
    to the winner.
    """
    import torch

    path = path or cache_path()
    gpu = torch.cuda.get_device_name()
    key = cache_key(gpu, policy, item_bytes, ranks, n, tag)
    shapes = rafi.rf_rounds_shapes(policy)
    if use_cache:
        hit = _load(path).get(key)
        if hit and 0 <= hit.get("shape", -1) < len(shapes) and hit.get("form") in forms:
            rafi.rf_set_batched_config(ctx, policy, hit["form"], hit["shape"])
            return {**hit, "cached": True, "key": key}
    s = stream or torch.cuda.current_stream()
    results = []
    for form, shape in candidates(policy, forms):
        rafi.rf_set_batched_config(ctx, policy, form, shape)
        try:
            run(form)  # warm-up: first launch of the shape, graph instantiation
        except rafi.RafiError as e:  # a shape this workload cannot use (too many digits for its block)
            results.append({"form": form, "shape": shape, "error": str(e)})
            continue
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            run(form)
        e1.record(s)
        torch.cuda.synchronize()
        results.append({"form": form, "shape": shape, "ms": e0.elapsed_time(e1) / reps})
    timed = [r for r in results if "ms" in r]
    if not timed:
        raise RuntimeError(f"autotune: no candidate ran for policy {policy}: {results}")
    best = min(timed, key=lambda r: r["ms"])
    rafi.rf_set_batched_config(ctx, policy, best["form"], best["shape"])
    threads, k, ctas = shapes[best["shape"]]
    out = {"form": best["form"], "shape": best["shape"], "threads": threads, "items_per_thread": k,
           "ctas_per_sm": ctas, "ms": best["ms"], "candidates": results}
    if use_cache:
        _store(path, key, out)
    return {**out, "cached": False, "key": key}
