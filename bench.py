"""Benchmark: device-local work forwarding on one GB300.

One step = the forwarding microbenchmark run to termination three times
(destinations uniform, Zipf s=1.1, 6-neighbour on a 4x4x4 torus): 2^24
64-byte items over 64 logical ranks, seed, exchange, then {work; exchange}
rounds until no item is active.  ``value`` counts items delivered by the
exchanges of work rounds (the seed exchange is timed but not counted) per
second of device time, for the batched form: the three runs in one
persistent kernel (rf_c1_run_batched_runs), every round of every run inside
it; each run keeps its own queues and retirement order, exactly those of a
launch of its own.  Inputs are resident in HBM before timing, and the
queues (3 GiB) are larger than L2.

Also reported on the same line: the persistent kernel's roofline
(algorithmic bytes over its CUDA-event time) and its per-round count and
scatter phase rates from its round log; the same runs as three separate
persistent launches (rf_c1_run_batched) with per-law times; the
step-in-place persistent form, the host loop's kernels in a CUDA graph and
the plain per-round host loop (rf_c1_run) with the scatter kernel's
roofline; the same step end to end through rf_c1_run_batched_runs with host
buffers; rays/s of the 64^3 marching workload; particle-steps/s of the
streamline workload (512^3 field, 16 uneven seed sets in one launch, batched
and plain forms); rays/s of the differentiable renderer (forward and
adjoint) and paths/s of the delta-tracking transport (1024^3, 512 ranks,
four views at 16 spp); the oracle timed on the host (cpu_baseline, one GPU
only): single-threaded on a bounded sample, on all host threads over the
whole microbenchmark, and on subsets of the streamline and transport
workloads; SM clocks sampled during the timed region and the number of
kernels launched.

``--impl reference`` times the oracle (the CPU reference of this method) on a
bounded sample of the same workload instead, on all host threads.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "forwarded items/s and rays/s on 1 GB300; forwarding HBM GB/s as % of peak"
N_ITEMS = 1 << 24
RANKS = 64
GRID = (4, 4, 4)
SEED = 1
ITEM_BYTES = 64
MODES = (0, 1, 2)  # uniform, Zipf 1.1, 6-neighbour torus
LAW_NAMES = {0: "uniform", 1: "zipf_1.1", 2: "torus_6"}
WORKLOAD = ("forwarding microbenchmark: 2^24 x 64-byte items (Philox payloads), 64 logical ranks, "
            "destinations uniform / Zipf s=1.1 / 6-neighbour 4x4x4 torus, retire p=0.1, seed 1; "
            "one step = the three runs, each seeded and run to zero active items")
SAMPLE_ITEMS = 1 << 21  # oracle sample per destination law, per reference-arm step (all host threads)
CPU_SAMPLE_ITEMS = 1 << 22  # single-thread oracle sample per destination law for cpu_baseline (about 5 s)
C2_ORACLE_SEEDS = 1 << 14  # streamline seeds the oracle traces for cpu_baseline
C4_ORACLE_CROP = 64  # 64 x 64 pixel crop of the first view the oracle renders for cpu_baseline


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.reader.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# the oracle on a bounded sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def host_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            lines = f.read().splitlines()
    except OSError:
        lines = []
    for key in ("model name", "CPU part"):
        for ln in lines:
            if ln.startswith(key) and ":" in ln:
                v = ln.split(":", 1)[1].strip()
                return v if key == "model name" else f"{platform.machine()}, CPU part {v}"
    return platform.machine()


def on_threads(fn, shards, threads):
    """fn over independent shards on `threads` host threads (the oracle's C calls
    release the GIL, so the shards run in parallel)."""
    if threads <= 1 or len(shards) <= 1:
        return [fn(x) for x in shards]
    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(fn, shards))


def oracle_sample_step(sample_items, threads=1):
    """Forwarded items of the three runs over sample_items.  With threads > 1 the
    items are split into contiguous shards of whole multiples of the rank count
    (item i keeps its start rank i mod 64); every item's hops depend on its own
    payload only, so the shards' forwarded counts add up to the whole sample's."""
    import oracle

    n = sample_items.shape[0]
    per = -(-n // max(threads, 1))
    per = max(RANKS, -(-per // RANKS) * RANKS)
    shards = [sample_items[a:a + per] for a in range(0, n, per)]

    def one(sh):
        f = 0
        for mode in MODES:
            res = oracle.c1_rounds(sh, RANKS, SEED, mode, grid=GRID)
            f += int(res["active"][1:].sum())
        return f

    return sum(on_threads(one, shards, threads))


def oracle_baseline(n=N_ITEMS):
    """The oracle on the host: single-threaded on 2^22 items per law (the parity
    oracle as it is), and on all host threads over the bench's n items per law."""
    from paper_2605_30294_gb300 import inputs

    items = inputs.c1_items(n, seed=SEED)
    t0 = time.perf_counter()
    fwd1 = oracle_sample_step(items[:CPU_SAMPLE_ITEMS])
    dt1 = time.perf_counter() - t0
    threads = host_threads()
    t0 = time.perf_counter()
    fwd = oracle_sample_step(items, threads)
    dt = time.perf_counter() - t0
    return {"value": fwd / dt, "unit": "items/s", "cores": threads, "kind": "oracle",
            "sample": f"the bench's workload ({n} items per destination law) split into {threads} shards "
                      f"run round by round through the oracle's queues, one host thread each, {dt:.1f} s",
            "cpu": cpu_model(),
            "single_thread": {"value": fwd1 / dt1, "unit": "items/s", "cores": 1,
                              "sample": f"{CPU_SAMPLE_ITEMS} items per destination law, {dt1:.1f} s"}}


def repeat_for(fn, min_s=1.0):
    """Runs fn until at least min_s seconds have passed; returns (fn's last result, runs, seconds)."""
    runs, t0 = 0, time.perf_counter()
    while True:
        r = fn()
        runs += 1
        dt = time.perf_counter() - t0
        if dt >= min_s:
            return r, runs, dt


def oracle_c2_subset(field, seeds, brick):
    """Streamline oracle on every k-th seed (C2_ORACLE_SEEDS of them), all host threads."""
    import oracle

    stride = max(1, seeds.shape[0] // C2_ORACLE_SEEDS)
    sub = np.ascontiguousarray(seeds[::stride][:C2_ORACLE_SEEDS])
    threads = host_threads()
    shards = np.array_split(sub, threads)
    steps, runs, dt = repeat_for(lambda: sum(
        int(r["steps"].astype(np.int64).sum())
        for r in on_threads(lambda x: oracle.c2_trace(field, x, brick), shards, threads)))
    return {"particle_steps_per_s": runs * steps / dt, "cores": threads, "kind": "oracle",
            "sample": f"subset: {sub.shape[0]} of {seeds.shape[0]} seeds (every {stride}th), "
                      f"{steps} particle-steps per run, {runs} runs in {dt:.1f} s"}


def oracle_c4_subset(vol, smax, view, spp):
    """Transport oracle on a centred crop of one view, all host threads (one band of rows each)."""
    import oracle

    cam, w, h, base = view
    c = C4_ORACLE_CROP
    x0, y0 = w // 2 - c // 2, h // 2 - c // 2
    threads = host_threads()
    bands = [(y0 + a[0], len(a)) for a in np.array_split(np.arange(c), threads) if len(a)]
    _, runs, dt = repeat_for(lambda: on_threads(
        lambda b: oracle.c4_render_crop(vol, smax, cam, w, base, x0, b[0], c, b[1], spp), bands, threads))
    return {"paths_per_s": runs * c * c * spp / dt, "cores": threads, "kind": "oracle",
            "sample": f"subset: the centred {c}x{c} crop of the {w}x{h} view at {spp} spp "
                      f"({c * c * spp} paths per run), {runs} runs in {dt:.1f} s"}


def reduce_over_ranks(dist, device, sec: float, units: int, e2e_s: float, e2e_units: int):
    """Replicas: the job's time is the slowest rank's, its work every rank's.
    Returns (max seconds, summed units, max end-to-end seconds, summed end-to-end units)."""
    import torch

    tt = torch.tensor([sec, float(units), e2e_s, float(e2e_units)], dtype=torch.float64, device=device)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = tt.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), int(sm[1]), float(mx[2]), int(sm[3])


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2605_30294_gb300 import inputs

    items = inputs.c1_items(SAMPLE_ITEMS, seed=SEED)
    threads = host_threads()
    for _ in range(args.warmup):
        oracle_sample_step(items, threads)
    t0 = time.perf_counter()
    fwd = 0
    for _ in range(args.steps):
        fwd += oracle_sample_step(items, threads)
    dt = time.perf_counter() - t0
    v = fwd / dt
    sample = (f"{SAMPLE_ITEMS} of the 2^24 items per destination law (same seed, ranks and laws), "
              f"run round by round through the oracle's queues in {threads} shards, one host thread each")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "items/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": "items/s", "cores": threads, "kind": "oracle", "sample": sample,
                             "cpu": cpu_model()},
            "e2e": {"value": v, "unit": "items/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the GPU path
# ---------------------------------------------------------------------------
def rounds_kernel_traffic():
    """DRAM bytes per full-size launch of the persistent kernel from the committed ncu
    summary, or None when the kernel's code changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "rounds_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    return d.get("bytes_per_full_size_launch") if d.get("code_sha256") == rounds_kernel_code_hash() else None


def rounds_kernel_code_hash() -> str:
    """sha256 of the persistent kernel's sources with comments and blank space
    removed (a change of comments leaves the captured counters valid)."""
    import hashlib
    import re

    srcs = ("paper_2605_30294_gb300/csrc/rounds.cuh", "paper_2605_30294_gb300/csrc/c1_microbench.cu")
    text = "".join(open(os.path.join(ROOT, x)).read() for x in srcs)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return hashlib.sha256(re.sub(r"\s+", "", text).encode()).hexdigest()


def sm_clock_mhz() -> float:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f).get("sm_max_mhz", 2070.0))
    return 2070.0


def l1_peak_gbs(torch) -> float:
    """Nominal L1 load bandwidth: 128 B per clock per SM at the SM clock."""
    return torch.cuda.get_device_properties(0).multi_processor_count * 128 * sm_clock_mhz() * 1e6 / 1e9


def issue_peak(torch) -> float:
    """Warp instructions per second: four schedulers per SM, one issue each per clock."""
    return torch.cuda.get_device_properties(0).multi_processor_count * 4 * sm_clock_mhz() * 1e6


def ea_march_instructions() -> dict:
    """Warp instructions of the EA march kernels per render at the configured size
    (profiles/ea_march_instructions.json), or {} when their code changed since."""
    import hashlib
    import re

    p = os.path.join(ROOT, "profiles", "ea_march_instructions.json")
    if not os.path.exists(p):
        return {}
    with open(p) as f:
        d = json.load(f)
    text = open(os.path.join(ROOT, "paper_2605_30294_gb300/csrc/c3_ea_render.cu")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    code = hashlib.sha256(re.sub(r"\s+", "", text).encode()).hexdigest()
    return d.get("warp_instructions", {}) if d.get("code_sha256") == code else {}


def c0_rays_per_s(torch, rafi, inputs, s, reps=20):
    n, w, h, brick = 64, 128, 128, 32
    vol = inputs.c0_volume(n)
    cam = inputs.c0_camera(n, w, h)
    dvol = torch.from_numpy(vol.reshape(-1)).cuda()
    bricks = torch.zeros(rafi.c0_bricks_floats(n, brick), dtype=torch.float32, device="cuda")
    rafi.rf_c0_make_bricks(dvol, n, brick, bricks, s)
    image = torch.zeros(w * h, dtype=torch.float32, device="cuda")
    sbricks = torch.zeros(rafi.c0_scalar_bricks_floats(n, brick), dtype=torch.float32, device="cuda")
    rafi.rf_c0_make_scalar_bricks(dvol, n, brick, sbricks, s)
    out = {}
    with rafi.Context(8, 48, w * h) as ctx:
        for name, render in (("host_loop", rafi.rf_c0_render), ("graph", rafi.rf_c0_render_graph),
                             ("tma", lambda c, b, *a, **k: rafi.rf_c0_render_tma(c, sbricks, *a, **k)),
                             ("tma_graph", lambda c, b, *a, **k: rafi.rf_c0_render_tma(c, sbricks, *a, **k,
                                                                                       form=rafi.RF_FORM_GRAPH))):
            for _ in range(3):
                render(ctx.handle, bricks, cam, n, brick, w, h, image, stream=s)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                render(ctx.handle, bricks, cam, n, brick, w, h, image, stream=s)
            e1.record(s)
            torch.cuda.synchronize()
            out[name] = e0.elapsed_time(e1) / reps
    return {k: {"value": w * h / (v * 1e-3), "ms_per_frame": v} for k, v in out.items()}


LOG_CAP = 4096  # rounds logged by the persistent kernel


def phase_rates(log_rows, item_bytes, min_items=1 << 20):
    """Per-round rates of the persistent kernel from its round log.

    Round 0 steps the seeded queue in place (read and write every item) and
    scatters it; every later round only counts the destinations of its
    already-stepped queue (4 bytes an item) before its scatter, which reads
    every queued item and writes it to its destination's segment, where the
    next round's step is applied on arrival, or to the retirement sink.  A
    phase lasts until the barrier that ends it completes, so the slowest CTA
    sets its time: count (or step) = round start -> first barrier done,
    scatter = first barrier done -> second barrier done.
    """
    lg = np.asarray(log_rows, dtype=np.float64)
    big = lg[:, 5] >= min_items
    first = np.arange(len(lg)) == 0
    work_b = np.where(first, lg[:, 5] * 2 * item_bytes, lg[:, 5] * 4)
    scat_b = lg[:, 5] * (2 * item_bytes + 4) + lg[:, 6] * 4
    work_t = (lg[:, 2] - lg[:, 0]) * 1e-9
    scat_t = (lg[:, 4] - lg[:, 2]) * 1e-9
    out = {"rounds": int(len(lg)), "rounds_ge_2^20": int(big.sum())}
    if big.any():
        later = big & ~first
        if later.any():
            out["count_us_per_round_ge_2^20"] = float(work_t[later].mean() * 1e6)
        out["scatter_gbs_ge_2^20"] = float(scat_b[big].sum() / scat_t[big].sum() / 1e9)
        per_round = scat_b[big] / scat_t[big] / 1e9
        out["scatter_gbs_ge_2^20_min_round"] = float(per_round.min())
        round_s = (lg[big, 4] - lg[big, 0]).sum() * 1e-9
        out["round_gbs_ge_2^20"] = float((work_b[big].sum() + scat_b[big].sum()) / round_s / 1e9)
        # forwarding rate in algorithmic bytes: 2 x itemBytes per item the round
        # forwards (its n_next), over the whole round, start to second barrier
        fwd_b = lg[:, 6] * 2 * item_bytes
        out["fwd_gbs_ge_2^20"] = float(fwd_b[big].sum() / round_s / 1e9)
        per_fwd = fwd_b[big] / ((lg[big, 4] - lg[big, 0]) * 1e-9) / 1e9
        out["fwd_gbs_ge_2^20_min_round"] = float(per_fwd.min())
    small = ~big
    if small.any():
        out["us_per_round_lt_2^20"] = float((lg[small, 4] - lg[small, 0]).mean() * 1e-3)
    # rounds of at most one 512-item tile run on one CTA; the ones between run on the whole grid
    for name, sel in (("solo_le_512", lg[:, 5] <= 512), ("grid_lt_2^20", small & (lg[:, 5] > 512)),
                      ("ge_2^20", big)):
        if sel.any():
            out["rounds_" + name] = int(sel.sum())
            out["us_per_round_" + name] = float((lg[sel, 4] - lg[sel, 0]).mean() * 1e-3)
            # as seen by CTA 0: count (or step), first barrier, offsets + scatter, second barrier
            out["us_split_" + name] = [float(x) for x in np.diff(lg[sel, :5], axis=1).mean(axis=0) * 1e-3]
    out["round_ms_total"] = float((lg[-1, 4] - lg[0, 0]) * 1e-6) if len(lg) else 0.0
    return out


def c2_streamlines(torch, rafi, inputs, s, reps=3, cpu=None):
    """Streamlines: 512^3 field over 4x4x4 ranks, the 16 uneven seed sets in one launch.

    Returns particle-steps/s and items forwarded/s of the batched (persistent)
    and plain (host loop) forms, CUDA events around each run.
    """
    n, brick = 512, 128
    R = (n // brick) ** 3
    field, _ = inputs.c2_field(n)
    sizes = inputs.c2_seed_set_sizes()
    count = sum(sizes)
    seeds = inputs.c2_seeds(count, n, seed=2)
    set_ids = np.repeat(np.arange(len(sizes), dtype=np.uint32), sizes)
    d_field = torch.from_numpy(field.reshape(-1)).cuda()
    bricks = torch.zeros(rafi.c2_bricks_floats(n, brick), dtype=torch.float32, device="cuda")
    rafi.rf_c2_make_bricks(d_field, n, brick, bricks, s)
    del d_field
    d_seeds = torch.from_numpy(seeds).cuda()
    d_sets = torch.from_numpy(set_ids.view(np.int32)).cuda()
    out = torch.zeros((count, 8), dtype=torch.int32, device="cuda")
    res = {"workload": f"512^3 curl-noise field (32 modes, |k| 1..8), 4x4x4 ranks of 128^3 bricks, "
                       f"{len(sizes)} uneven seed sets ({sizes[0]}..{sizes[-1]}, {count} particles) in one launch, "
                       f"RK4 h=0.25, <= 2000 steps",
           "particles": count}
    from paper_2605_30294_gb300 import autotune

    # the autotuner times the workload itself (a quarter of the particles picked
    # a shape that lost at full size: occupancy matters less with fewer particles)
    with rafi.Context(R, 32, count) as ctx:
        # steps per round: 0 = until a particle leaves its brick; 1 = the paper's
        # pattern (one RK step per round, every particle forwarded every round)
        for spr, nrep in ((0, reps), (1, 1)):
            key = "brick_exit" if spr == 0 else "one_step_per_round"
            res[key] = {}

            def sample(form, spr=spr):
                rafi.rf_c2_run(ctx.handle, bricks, d_seeds, d_sets, count, n, brick, 0.25, 2000, spr, out,
                               rafi.RF_FORM_TUNED, stream=s)

            res[key]["autotune"] = autotune.tune(
                ctx.handle, rafi.RF_POLICY_STREAMLINES, sample, item_bytes=32, ranks=R, n=count,
                tag=f"steps_per_round={spr}", forms=(rafi.RF_FORM_HOST_LOOP, rafi.RF_FORM_PERSISTENT,
                                                      rafi.RF_FORM_GRAPH), reps=1, stream=s)
            res[key]["autotune"]["sample"] = f"the whole workload ({count} particles)"
            for batched in (rafi.RF_FORM_PERSISTENT, rafi.RF_FORM_HOST_LOOP, rafi.RF_FORM_GRAPH, rafi.RF_FORM_TUNED):
                if batched == rafi.RF_FORM_PERSISTENT:
                    rafi.rf_set_batched_config(ctx.handle, rafi.RF_POLICY_STREAMLINES, rafi.RF_FORM_PERSISTENT, 0)
                elif batched == rafi.RF_FORM_TUNED:
                    t = res[key]["autotune"]
                    rafi.rf_set_batched_config(ctx.handle, rafi.RF_POLICY_STREAMLINES, t["form"], t["shape"])
                for _ in range(2 if spr == 0 else 1):
                    rafi.rf_c2_run(ctx.handle, bricks, d_seeds, d_sets, count, n, brick, 0.25, 2000, spr, out,
                                   batched, stream=s)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                fwd = rounds = 0
                for _ in range(nrep):
                    st, rounds, f = rafi.rf_c2_run(ctx.handle, bricks, d_seeds, d_sets, count, n, brick, 0.25, 2000,
                                                   spr, out, batched, stream=s)
                    fwd += f
                e1.record(s)
                torch.cuda.synchronize()
                sec = e0.elapsed_time(e1) / 1e3 / nrep
                steps = int(out[:, 4].cpu().numpy().view(np.uint32).astype(np.int64).sum())
                res[key][("plain", "batched", "graph", "tuned")[batched]] = {
                    "ms_per_run": sec * 1e3, "particle_steps_per_s": steps / sec,
                    "items_forwarded_per_s": fwd / nrep / sec, "rounds": rounds, "particle_steps": steps}
            res[key]["batched_over_plain"] = res[key]["plain"]["ms_per_run"] / res[key]["batched"]["ms_per_run"]
            res[key]["graph_over_plain"] = res[key]["plain"]["ms_per_run"] / res[key]["graph"]["ms_per_run"]
            res[key]["tuned_over_plain"] = res[key]["plain"]["ms_per_run"] / res[key]["tuned"]["ms_per_run"]
            if spr == 0:
                # the trace kernel's L1 roofline: an RK4 step samples the velocity four
                # times, each sample four aligned 32-byte loads of x-paired voxels
                rafi.rf_set_timing(ctx.handle, True)
                rafi.rf_get_timing(ctx.handle, reset=True)
                rafi.rf_c2_run(ctx.handle, bricks, d_seeds, d_sets, count, n, brick, 0.25, 2000, spr, out,
                               rafi.RF_FORM_HOST_LOOP, stream=s)
                t = rafi.rf_get_timing(ctx.handle, reset=True)
                rafi.rf_set_timing(ctx.handle, False)
                steps = res[key]["plain"]["particle_steps"]
                achieved = steps * 512 / (t.workMs * 1e-3) / 1e9
                peak = l1_peak_gbs(torch)
                res[key]["roofline_trace"] = {
                    "bound": "l1", "kernel": "trace_kernel", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "kernel_ms": t.workMs, "launches": t.workLaunches,
                    "alg_bytes": "512 B per particle-step (4 samples x 4 loads x 32 B, from L1)",
                    "peak_kind": "derived: SMs x 128 B per clock x the SM clock"}
    if cpu is not None:  # the cpu_baseline leg: the oracle on a subset of the seeds
        cpu["streamlines_subset"] = oracle_c2_subset(field, seeds, brick)
    return res


def c3_ea(torch, rafi, inputs, s, reps=5):
    """Differentiable EA renderer: 256^3 over 2x2x2 ranks, 512x512 at 4 spp; forward and adjoint rays/s."""
    from paper_2605_30294_gb300 import ea_autograd  # noqa: F401  (the autograd wrapper uses the same calls)

    n, brick, w, h, spp = 256, 128, 512, 512, 4
    vol = inputs.c0_volume(n)
    cam = inputs.c0_camera(n, w, h)
    dv = torch.from_numpy(vol.reshape(-1)).cuda()
    bricks = torch.zeros(rafi.c0_bricks_floats(n, brick), dtype=torch.float32, device="cuda")
    rafi.rf_c0_make_bricks(dv, n, brick, bricks, s)
    nr = w * h * spp
    rayC = torch.zeros(nr, dtype=torch.float32, device="cuda")
    rayClo = torch.zeros(nr, dtype=torch.float32, device="cuda")
    img = torch.zeros(w * h, dtype=torch.float32, device="cuda")
    gimg = torch.ones(w * h, dtype=torch.float32, device="cuda")
    grad = torch.zeros(n ** 3, dtype=torch.float32, device="cuda")
    out = {"workload": "256^3 blob density, 2x2x2 ranks of 128^3, 512x512 at 4 spp (1,048,576 rays); forward "
                       "and adjoint as the autograd wrapper runs them (compensated colour sums)"}
    with rafi.Context(8, 64, nr) as ctx:
        for name, fn in (("forward", lambda: rafi.rf_c3_render(ctx.handle, bricks, cam, n, brick, w, h, spp, 3,
                                                                rayC, img, stream=s, ray_c_lo=rayClo)),
                         ("adjoint", lambda: rafi.rf_c3_adjoint(ctx.handle, bricks, cam, n, brick, w, h, spp, 3,
                                                                 rayC, gimg, grad, stream=s, ray_c_lo=rayClo))):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                fn()
            e1.record(s)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            out[name] = {"ms": ms, "rays_per_s": nr / (ms * 1e-3)}
            # the march kernels issue-bound roofline: their warp instructions (counted once
            # by ncu at this size) over their time in one more render
            rafi.rf_set_timing(ctx.handle, True)
            rafi.rf_get_timing(ctx.handle, reset=True)
            fn()
            t = rafi.rf_get_timing(ctx.handle, reset=True)
            rafi.rf_set_timing(ctx.handle, False)
            inst = ea_march_instructions().get(name)
            peak = issue_peak(torch)
            ach = inst / (t.workMs * 1e-3) if inst else None
            out[name]["roofline"] = {
                "bound": "issue", "kernel": f"march_kernel ({name})", "achieved": ach, "peak": peak,
                "unit": "warp instructions/s", "frac": ach / peak if ach else None, "kernel_ms": t.workMs,
                "warp_instructions": inst, "peak_kind": "derived: SMs x 4 schedulers x 1 warp instruction per clock "
                                                        "x the SM clock",
                "instructions_from": "profiles/ea_march_instructions.json (null when the kernel's code changed)"}
    return out


def c4_transport(torch, rafi, inputs, s, cpu=None):
    """Delta tracking: 1024^3 noise (mean optical depth 8) over 8x8x8 ranks, 4 views at 16 spp."""
    n, brick, spp = 1024, 128, 16
    vol, smax = inputs.c4_volume(n)
    views = inputs.c4_views(n)
    bricks = torch.zeros(rafi.c0_bricks_floats(n, brick), dtype=torch.float32, device="cuda")
    dv = torch.from_numpy(vol.reshape(-1)).cuda()
    rafi.rf_c0_make_bricks(dv, n, brick, bricks, s)
    del dv
    torch.cuda.empty_cache()
    npix = sum(w * h for _, w, h, _ in views)
    paths = npix * spp
    score = torch.zeros(npix, dtype=torch.float32, device="cuda")
    out = {"workload": "1024^3 fractal gradient noise (6 octaves), mean optical depth 8, 8x8x8 ranks of 128^3, "
                       "views 2048^2, 1024x768, 512^2, 3840x2160 at 16 spp, albedo 0.8, HG g=0.3, <= 64 bounces",
           "paths": paths}
    from paper_2605_30294_gb300 import autotune

    with rafi.Context(512, 64, paths) as ctx:
        # the autotuner times the workload itself: the four views at 16 spp
        def sample(form):
            rafi.rf_c4_render(ctx.handle, bricks, n, brick, smax, views, spp, 4, score, rafi.RF_FORM_TUNED,
                              stream=s)

        out["autotune"] = autotune.tune(ctx.handle, rafi.RF_POLICY_TRANSPORT, sample, item_bytes=64, ranks=512,
                                        n=paths, tag="four views", forms=(rafi.RF_FORM_HOST_LOOP,
                                                                          rafi.RF_FORM_PERSISTENT,
                                                                          rafi.RF_FORM_GRAPH), reps=1, stream=s)
        out["autotune"]["sample"] = f"the whole workload ({paths} paths)"
        for batched in (rafi.RF_FORM_PERSISTENT, rafi.RF_FORM_HOST_LOOP, rafi.RF_FORM_GRAPH, rafi.RF_FORM_TUNED):
            if batched == rafi.RF_FORM_PERSISTENT:
                rafi.rf_set_batched_config(ctx.handle, rafi.RF_POLICY_TRANSPORT, rafi.RF_FORM_PERSISTENT, 0)
            elif batched == rafi.RF_FORM_TUNED:
                rafi.rf_set_batched_config(ctx.handle, rafi.RF_POLICY_TRANSPORT, out["autotune"]["form"],
                                           out["autotune"]["shape"])
            score.zero_()
            rafi.rf_c4_render(ctx.handle, bricks, n, brick, smax, views, spp, 4, score, batched, stream=s)
            score.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            rounds, fwd = rafi.rf_c4_render(ctx.handle, bricks, n, brick, smax, views, spp, 4, score, batched,
                                            stream=s)
            e1.record(s)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            out[("plain", "batched", "graph", "tuned")[batched]] = {"ms": sec * 1e3, "paths_per_s": paths / sec,
                                                                     "rays_forwarded_per_s": fwd / sec,
                                                                     "rounds": rounds}
    out["batched_over_plain"] = out["plain"]["ms"] / out["batched"]["ms"]
    out["graph_over_plain"] = out["plain"]["ms"] / out["graph"]["ms"]
    out["tuned_over_plain"] = out["plain"]["ms"] / out["tuned"]["ms"]
    if cpu is not None:  # the cpu_baseline leg: the oracle on a crop of the first view
        cpu["transport_subset"] = oracle_c4_subset(vol, smax, views[0], spp)
    return out


def multi_phase(torch, rafi, inputs, s, n=1 << 22, steps=5):
    """Three contexts on one stream (particles 32 B, nodes 64 B, requests 16 B): one step =
    migrate + exchange, local trees, root broadcast + exchange, requests + exchange,
    replies + exchange (rf_mp_step, which reads each exchange's count back)."""
    grid, R = (4, 4, 4), 64
    p = inputs.mp_particles(n, seed=5)
    nodes = torch.zeros((R, 9, 5), dtype=torch.int64, device="cuda")
    with rafi.Context(R, 32, n) as pc, rafi.Context(R, 64, R * (R - 1) + R * 26 * 8) as nc, \
            rafi.Context(R, 16, R * 26) as rc:
        rafi.rf_mp_seed(pc.handle, torch.from_numpy(p.view(np.int32)).cuda(), n, grid, stream=s)
        rafi.rf_exchange(pc.handle, s)
        for _ in range(2):
            rafi.rf_mp_step(pc.handle, nc.handle, rc.handle, grid, nodes, stream=s)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        delivered = 0
        e0.record(s)
        for _ in range(steps):
            delivered += sum(rafi.rf_mp_step(pc.handle, nc.handle, rc.handle, grid, nodes, stream=s))
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
    return {"workload": f"{n} particles, 4x4x4 ranks, velocities up to 2^-6 of the cube per step",
            "ms_per_step": ms, "particles_per_s": n / (ms * 1e-3),
            "items_delivered_per_s": delivered / steps / (ms * 1e-3)}


def run_ours(args):
    import torch

    from paper_2605_30294_gb300 import build, inputs, rafi

    world, rank, local = dist_env()
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    n = args.items
    items = inputs.c1_items(n, seed=SEED)
    d_items = torch.from_numpy(items.view(np.int32)).to(dev)
    # the three runs of a step hold the same seeded items (one copy per run for
    # the joint launch, whose run k reads items [k n, (k + 1) n))
    d_items3 = torch.cat([d_items] * len(MODES))
    retired = torch.zeros((len(MODES) * n, 16), dtype=torch.int32, device=dev)
    log = torch.zeros(7 * LOG_CAP, dtype=torch.int64, device=dev)
    s = torch.cuda.current_stream(dev)
    ctx = rafi.Context(RANKS, ITEM_BYTES, n)  # one run at a time
    ctx3 = rafi.Context(RANKS, ITEM_BYTES, len(MODES) * n)  # the three runs in one launch

    def joint(round_log=None):
        # one step: the three runs in one persistent launch
        st, cnt, rounds, f = rafi.rf_c1_run_batched_runs(ctx3.handle, d_items3, n, SEED, list(MODES), 1.1, GRID,
                                                         retired, stream=s, round_log=round_log,
                                                         round_log_cap=LOG_CAP if round_log is not None else 0)
        if cnt != [n] * len(MODES):
            raise RuntimeError(f"joint runs: {cnt} of {n} items retired per run")
        return f

    def step(batched, round_log=None, fuse=True, per_mode=None):
        if batched == "joint":
            return joint(round_log)
        fwd = 0
        for mode in MODES:
            if per_mode is not None:
                ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                ev[0].record(s)
            if batched == "graph":
                st, cnt, rounds, f = rafi.rf_c1_run_graph(ctx.handle, d_items, n, SEED, mode, 1.1, GRID, retired,
                                                          stream=s)
            elif batched:
                st, cnt, rounds, f = rafi.rf_c1_run_batched(ctx.handle, d_items, n, SEED, mode, 1.1, GRID, retired,
                                                            stream=s, round_log=round_log,
                                                            round_log_cap=LOG_CAP if round_log is not None else 0,
                                                            step_on_arrival=fuse)
            else:
                st, cnt, rounds, f = rafi.rf_c1_run(ctx.handle, d_items, n, SEED, mode, 1.1, GRID, retired,
                                                    stream=s)
            if cnt != n:
                raise RuntimeError(f"mode {mode}: {cnt} of {n} items retired")
            if per_mode is not None:
                ev[1].record(s)
                per_mode.setdefault(mode, []).append((ev, f))
            fwd += f
        return fwd

    def timed(batched, steps, fuse=True):
        c = ctx3 if batched == "joint" else ctx
        rafi.rf_set_timing(c.handle, True)
        rafi.rf_get_timing(c.handle, reset=True)
        barrier()
        launches0 = rafi.rf_launch_count()
        per_mode = {}
        with ClockSampler(gpu_id) as clocks:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fwd = 0
            for _ in range(steps):
                fwd += step(batched, fuse=fuse, per_mode=per_mode)
            e1.record(s)
            barrier()
        launches = rafi.rf_launch_count() - launches0
        t = rafi.rf_get_timing(c.handle, reset=True)
        rafi.rf_set_timing(c.handle, False)
        # per destination law: ms per run and forwarded items/s (events around each run)
        laws = {}
        for mode, runs in per_mode.items():
            ms_law = sum(ev[0].elapsed_time(ev[1]) for ev, _ in runs)
            f_law = sum(f for _, f in runs)
            laws[LAW_NAMES[mode]] = {"ms_per_run": ms_law / len(runs), "items_per_s": f_law / (ms_law * 1e-3)}
        timed.laws = laws
        return fwd, e0.elapsed_time(e1), t, launches, clocks.summary()

    # the autotuner picks the persistent kernel's shape on one step of the workload itself
    from paper_2605_30294_gb300 import autotune

    tuned_c1 = autotune.tune(ctx3.handle, rafi.RF_POLICY_MICROBENCH, lambda form: joint(), item_bytes=ITEM_BYTES,
                             ranks=RANKS, n=len(MODES) * n, tag="three laws in one launch, steps on arrival",
                             reps=1, stream=s)
    # the separate launches run in the same shape
    rafi.rf_set_batched_config(ctx.handle, rafi.RF_POLICY_MICROBENCH, rafi.RF_FORM_PERSISTENT, tuned_c1["shape"])

    props = torch.cuda.get_device_properties(dev)
    gpu_id = None
    uuid = getattr(props, "uuid", None)
    if uuid is not None:
        gpu_id = str(uuid) if str(uuid).startswith("GPU-") else "GPU-" + str(uuid)

    for _ in range(args.warmup):
        joint()
        step(True)
        step(False)
    fwd, ms, tb, launches, clocks = timed("joint", args.steps)
    p_steps = max(3, args.steps // 4)
    # the same three runs, one persistent launch each
    sep_steps = max(3, args.steps // 2)
    s_fwd, s_ms, ts, s_launches, s_clocks = timed(True, sep_steps)
    laws_batched = timed.laws
    p_fwd, p_ms, tp, p_launches, p_clocks = timed(False, p_steps)
    # the persistent form with the work step as its own pass (no step on arrival)
    step(True, fuse=False)
    u_fwd, u_ms, tu, _, _ = timed(True, p_steps, fuse=False)
    laws_in_place = timed.laws
    # the host loop's rounds in a CUDA graph (conditional while node)
    step("graph")
    g_fwd, g_ms, _, g_launches, _ = timed("graph", p_steps)
    laws_graph = timed.laws

    # per-round phase rates of the persistent kernel (one extra, untimed step
    # of each form)
    def round_rates(form):
        log.zero_()
        step(form, round_log=log)
        lg = log.cpu().numpy().reshape(-1, 7)
        return phase_rates([r for r in lg if r[0] > 0], ITEM_BYTES)

    rates = round_rates("joint")
    rates_sep = round_rates(True)

    # end to end through the public call with host buffers (H2D + D2H inside)
    h_items = torch.empty((len(MODES) * n, 16), dtype=torch.int32).pin_memory()
    h_items.copy_(d_items3)
    h_ret = torch.zeros((len(MODES) * n, 16), dtype=torch.int32).pin_memory()

    def e2e_step():
        st, cnt, rounds, f = rafi.rf_c1_run_batched_runs(ctx3.handle, h_items.data_ptr(), n, SEED, list(MODES), 1.1,
                                                         GRID, h_ret.data_ptr(), host_memory=True, stream=s)
        if cnt != [n] * len(MODES):
            raise RuntimeError(f"joint runs from host buffers: {cnt} of {n} items retired per run")
        return f

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    e2e_fwd = 0
    e2e_steps = max(1, min(args.steps, 10))
    e2e_step_ms = []
    for _ in range(e2e_steps):
        t1 = time.perf_counter()
        e2e_fwd += e2e_step()  # returns after the stream has drained
        e2e_step_ms.append((time.perf_counter() - t1) * 1e3)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_fwd_rank = e2e_fwd

    # where the end-to-end time goes: one more step with the persistent kernel
    # timed on the device (it writes the retired items straight into the pinned
    # host buffer), and the host-to-device copy of one step's items timed alone
    rafi.rf_set_timing(ctx3.handle, True)
    rafi.rf_get_timing(ctx3.handle, reset=True)
    barrier()
    t0 = time.perf_counter()
    e2e_step()
    barrier()
    one_step_s = time.perf_counter() - t0
    te = rafi.rf_get_timing(ctx3.handle, reset=True)
    rafi.rf_set_timing(ctx3.handle, False)
    # one run's items (1 GiB) copied in alone, five times: the median (the
    # shared hosts' link now and then stalls a copy for a hundred ms or more)
    retired[:n].copy_(h_items[:n], non_blocking=True)  # first copy: untimed
    copy_ms = []
    for _ in range(5):
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record(s)
        retired[:n].copy_(h_items[:n], non_blocking=True)
        ev[1].record(s)
        torch.cuda.synchronize()
        copy_ms.append(ev[0].elapsed_time(ev[1]))
    first_copy_ms = statistics.median(copy_ms)
    step_ms = one_step_s * 1e3
    kern_ms = te.roundsMs  # the step's persistent launches, one per run
    e2e_split = {"ms_per_step": step_ms, "h2d_run_ms": [round(x, 3) for x in copy_ms],
                 "h2d_gbs": n * ITEM_BYTES / (first_copy_ms * 1e-3) / 1e9,
                 "first_run_copy_ms": first_copy_ms,
                 "rounds_kernel_ms": kern_ms, "rounds_kernel_launches": te.roundsLaunches,
                 "rounds_kernel_ms_device_buffers": tb.roundsMs / max(tb.roundsLaunches, 1),
                 "rest_ms": step_ms - first_copy_ms - kern_ms,
                 "what": "one step = the first run's items copied in, then per run its seed kernel and persistent "
                         "kernel (writing its retired items into the pinned host buffer) while the next run's "
                         "items are copied in on a second stream, read-back of the counts; h2d_run_ms: one run's "
                         "copy timed alone (first_run_copy_ms: their median); rest = launches, host calls, "
                         "waits for a copy and synchronisation"}

    c0 = c0_rays_per_s(torch, rafi, inputs, s)
    ctx.close()
    ctx3.close()
    del d_items, d_items3, retired, h_items, h_ret
    torch.cuda.empty_cache()
    # the oracle's timings (cpu_baseline) run at one GPU only
    cpu_extra = {} if world == 1 else None
    streamlines = c2_streamlines(torch, rafi, inputs, s, cpu=cpu_extra) if not args.skip_extra else None
    torch.cuda.empty_cache()
    ea = c3_ea(torch, rafi, inputs, s) if not args.skip_extra else None
    torch.cuda.empty_cache()
    transport = c4_transport(torch, rafi, inputs, s, cpu=cpu_extra) if not args.skip_extra else None
    torch.cuda.empty_cache()
    mp = multi_phase(torch, rafi, inputs, s) if not args.skip_extra else None

    sec = ms / 1e3
    total_fwd = fwd
    if pg:
        sec, total_fwd, e2e_s, e2e_fwd = reduce_over_ranks(pg, dev, sec, fwd, e2e_s, e2e_fwd)
    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0

    peak, peak_kind = peaks()
    # persistent kernel, algorithmic bytes as the forwarding layer counts them:
    # 2 x itemBytes per forwarded item (an item delivered by a work round's
    # exchange), so `fwd` items move 128 * fwd bytes over all timed launches.
    # Also reported: the bytes the kernel actually has to move, the queued
    # items of every round (each read once and written once, to its next
    # segment or to the retirement sink) plus the seed exchange's items (3 n
    # per joint launch, n per separate one).
    runs = tb.roundsLaunches
    alg_bytes = 2 * ITEM_BYTES * fwd
    achieved = alg_bytes / (tb.roundsMs * 1e-3) / 1e9 if tb.roundsMs > 0 else 0.0
    moved_bytes = 2 * ITEM_BYTES * (2 * runs * len(MODES) * n + fwd)
    moved = moved_bytes / (tb.roundsMs * 1e-3) / 1e9 if tb.roundsMs > 0 else 0.0
    s_runs = ts.roundsLaunches
    s_ach = 2 * ITEM_BYTES * s_fwd / (ts.roundsMs * 1e-3) / 1e9 if ts.roundsMs > 0 else 0.0
    s_moved = 2 * ITEM_BYTES * (2 * s_runs * n + s_fwd) / (ts.roundsMs * 1e-3) / 1e9 if ts.roundsMs > 0 else 0.0
    p_bytes = tp.scatterItems * 2 * ITEM_BYTES
    p_ach = p_bytes / (tp.scatterMs * 1e-3) / 1e9 if tp.scatterMs > 0 else 0.0
    p_ach_l = (tp.scatterItemsLarge * 2 * ITEM_BYTES / (tp.scatterMsLarge * 1e-3) / 1e9
               if tp.scatterMsLarge > 0 else 0.0)
    u_ach = (2 * ITEM_BYTES * (tu.roundsLaunches * n + 2 * u_fwd) / (tu.roundsMs * 1e-3) / 1e9
             if tu.roundsMs > 0 else 0.0)
    cpu_line = None
    if cpu_extra is not None:
        cpu_line = oracle_baseline(n)
        cpu_line.update(cpu_extra)
    line = {
        "metric": METRIC, "value": total_fwd / sec, "unit": "items/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "items": n, "item_bytes": ITEM_BYTES, "ranks": RANKS,
                   "form": "batched: the three runs (laws) of a step in one persistent cooperative kernel "
                           "(rf_c1_run_batched_runs), all their rounds inside it, each step applied on arrival; "
                           "each run's queues and retirements are those of its own launch",
                   "shape": {"threads": tuned_c1["threads"], "items_per_thread": tuned_c1["items_per_thread"],
                             "ctas_per_sm": tuned_c1["ctas_per_sm"], "chosen_by": "autotune"},
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "no flush: the 1 GiB item queues exceed the 129 MB L2"},
        "roofline": {"bound": "hbm", "kernel": "rounds_kernel<C1Work>", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": rounds_kernel_traffic(),
                     "peak_kind": peak_kind,
                     "alg_bytes": "2 x 64 B per forwarded item (deliveries of work rounds)",
                     "alg_bytes_per_launch": alg_bytes / max(runs, 1), "launches": runs,
                     "ms_total": tb.roundsMs, "ms_per_launch": tb.roundsMs / max(runs, 1),
                     "frac_rounds_ge_2^20": rates.get("fwd_gbs_ge_2^20", 0.0) / peak,
                     "moved": {"bytes_per_launch": moved_bytes / max(runs, 1), "achieved": moved,
                               "frac": moved / peak,
                               "what": "2 x 64 B per queued item of every round plus the seed exchange"}},
        "phases_from_round_log": {**rates,
                                  "scatter_frac_ge_2^20": rates.get("scatter_gbs_ge_2^20", 0.0) / peak,
                                  "round_frac_ge_2^20": rates.get("round_gbs_ge_2^20", 0.0) / peak,
                                  "fwd_frac_ge_2^20": rates.get("fwd_gbs_ge_2^20", 0.0) / peak},
        "autotune": tuned_c1,
        "separate_launches": {
            "value": s_fwd / (s_ms / 1e3), "ms_per_step": s_ms / sep_steps, "steps": sep_steps,
            "per_law": laws_batched, "gpu_launches": s_launches, "clocks": s_clocks,
            "form": "the same persistent kernel, one launch per run (rf_c1_run_batched, steps on arrival)",
            "roofline": {"achieved": s_ach, "frac": s_ach / peak, "launches": s_runs,
                         "ms_per_launch": ts.roundsMs / max(s_runs, 1),
                         "frac_rounds_ge_2^20": rates_sep.get("fwd_gbs_ge_2^20", 0.0) / peak,
                         "moved_frac": s_moved / peak},
            "phases_from_round_log": rates_sep},
        "batched_step_in_place": {
            "value": u_fwd / (u_ms / 1e3), "ms_per_step": u_ms / p_steps, "steps": p_steps, "per_law": laws_in_place,
            "form": "persistent kernel; each round steps every item in its queue slot, then scatters",
            "roofline": {"achieved": u_ach, "frac": u_ach / peak,
                         "alg_bytes": "2 x 64 B per queued item for the step pass, 2 x 64 B per delivery"}},
        "graph_loop": {"value": g_fwd / (g_ms / 1e3), "ms_per_step": g_ms / p_steps, "steps": p_steps,
                       "per_law": laws_graph, "gpu_launches": g_launches,
                       "form": "the host loop's kernels captured once into a CUDA graph whose conditional "
                               "while node repeats them on the device"},
        "plain": {"value": p_fwd / (p_ms / 1e3), "ms_per_step": p_ms / p_steps, "steps": p_steps,
                  "form": "host loop: work kernel + count/scan/scatter/wrap-up kernels + one sync per round",
                  "roofline_scatter": {"achieved": p_ach, "frac": p_ach / peak,
                                       "achieved_rounds_ge_2^20": p_ach_l, "frac_rounds_ge_2^20": p_ach_l / peak,
                                       "launches": tp.scatterLaunches},
                  "phase_ms": {"work": tp.workMs, "count": tp.countMs, "scan": tp.scanMs,
                               "scatter": tp.scatterMs},
                  "gpu_launches": p_launches, "clocks": p_clocks},
        "e2e": {"value": e2e_fwd / e2e_s, "unit": "items/s",
                "h2d_bytes_per_step": len(MODES) * n * ITEM_BYTES,
                "d2h_bytes_per_step": len(MODES) * (n * ITEM_BYTES + 8), "steps": e2e_steps,
                "step_ms": [round(x, 3) for x in e2e_step_ms],
                "value_at_median_step": world * (e2e_fwd_rank / e2e_steps) / (statistics.median(e2e_step_ms) * 1e-3),
                "split": e2e_split,
                "note": "the host link of the shared GPU hosts carries other jobs' copies too: step_ms shows "
                        "the spread"},
        "rays_per_s": {"value": c0["tma_graph"]["value"],
                       "workload": "64^3 blob volume, 2x2x2 ranks, 128x128 rays, 1 spp",
                       "ms_per_frame": c0["tma_graph"]["ms_per_frame"],
                       "form": "bricks staged whole in shared memory by one 3-D tensor copy, rounds in a kept CUDA "
                               "graph (rf_c0_render_tma, graph form)",
                       "forms": {"quad_bricks_host_loop": c0["host_loop"], "quad_bricks_graph": c0["graph"],
                                 "tma_bricks_host_loop": c0["tma"], "tma_bricks_graph": c0["tma_graph"]}},
        "streamlines": streamlines,
        "differentiable_ea": ea,
        "delta_tracking": transport,
        "multi_phase": mp,
        "cpu_baseline": cpu_line,
        "clocks": clocks,
        "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def run_section(args):
    """One workload alone, at a size for a profiler capture (a few GB on the
    device, each workload launched once, no warm-up), printing one JSON line of
    its own (not the bench line):
      c0: the marching workload, one frame with quad bricks, one with TMA-staged bricks;
      c1: the microbenchmark, one rf_c1_run_batched call (one persistent launch),
          or with --joint one rf_c1_run_batched_runs call of the three laws;
      c2: streamlines, 512^3 field in 4x4x4 bricks, 2^18 seeds, until brick exit;
      c3: EA renderer at its configured size, one forward and one adjoint render;
      c4: delta tracking, 512^3 noise in 4x4x4 bricks, one 512x512 view at 16 spp."""
    import torch

    from paper_2605_30294_gb300 import build, inputs, rafi

    build.build()
    torch.cuda.set_device(0)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"section": args.section}
    if args.section == "c1":
        # one persistent-kernel launch of the microbenchmark (steps on arrival),
        # one destination law, no warm-up: the launch a profiler captures
        n = args.items
        k = len(MODES) if args.joint else 1
        items = inputs.c1_items(n, seed=SEED)
        d_items = torch.cat([torch.from_numpy(items.view(np.int32)).cuda()] * k)
        retired = torch.zeros((k * n, 16), dtype=torch.int32, device="cuda")
        log = torch.zeros(7 * LOG_CAP, dtype=torch.int64, device="cuda")
        with rafi.Context(RANKS, ITEM_BYTES, k * n) as ctx:
            e0.record(s)
            if args.joint:
                st, cnt, rounds, fwd = rafi.rf_c1_run_batched_runs(ctx.handle, d_items, n, SEED, list(MODES), 1.1,
                                                                   GRID, retired, stream=s, round_log=log,
                                                                   round_log_cap=LOG_CAP)
            else:
                st, cnt, rounds, fwd = rafi.rf_c1_run_batched(ctx.handle, d_items, n, SEED, args.law, 1.1, GRID,
                                                              retired, stream=s, round_log=log, round_log_cap=LOG_CAP)
            e1.record(s)
            torch.cuda.synchronize()
        lg = log.cpu().numpy().reshape(-1, 7)
        rows = [r for r in lg if r[0] > 0]
        what = ("the three laws in one rf_c1_run_batched_runs call" if args.joint else
                f"law {LAW_NAMES[args.law]}, one rf_c1_run_batched call")
        out.update(workload=f"microbenchmark, {n} x 64 B items per run, 64 ranks, {what}", items=k * n,
                   ms=e0.elapsed_time(e1), rounds=rounds, forwarded=fwd, retired=cnt,
                   phases=phase_rates(rows, ITEM_BYTES))
        if args.round_log:
            with open(args.round_log, "w") as f:
                json.dump({"columns": ["t_start", "t_count_end", "t_barrier1", "t_scatter_end", "t_barrier2",
                                       "n_in", "n_next"], "rows": [[int(x) for x in r] for r in rows]}, f)
    elif args.section == "c0":
        # the marching workload once with quad bricks read through L1 and once
        # with each brick staged whole in shared memory by a tensor copy
        n, w, h, brick = 64, 128, 128, 32
        vol = inputs.c0_volume(n)
        cam = inputs.c0_camera(n, w, h)
        dvol = torch.from_numpy(vol.reshape(-1)).cuda()
        bricks = torch.zeros(rafi.c0_bricks_floats(n, brick), dtype=torch.float32, device="cuda")
        rafi.rf_c0_make_bricks(dvol, n, brick, bricks, s)
        sbricks = torch.zeros(rafi.c0_scalar_bricks_floats(n, brick), dtype=torch.float32, device="cuda")
        rafi.rf_c0_make_scalar_bricks(dvol, n, brick, sbricks, s)
        image = torch.zeros(w * h, dtype=torch.float32, device="cuda")
        out["workload"] = "64^3 blob volume, 2x2x2 ranks of 32^3, 128x128 rays, one frame each way"
        with rafi.Context(8, 48, w * h) as ctx:
            for name, fn in (("quad_l1", lambda: rafi.rf_c0_render(ctx.handle, bricks, cam, n, brick, w, h, image,
                                                                    stream=s)),
                             ("tma_smem", lambda: rafi.rf_c0_render_tma(ctx.handle, sbricks, cam, n, brick, w, h,
                                                                         image, stream=s))):
                e0.record(s)
                rounds = fn()
                e1.record(s)
                torch.cuda.synchronize()
                out[name] = {"ms": e0.elapsed_time(e1), "rounds": rounds}
    elif args.section == "c2":
        n, brick, count = 512, 128, 1 << 18
        R = (n // brick) ** 3
        field, _ = inputs.c2_field(n)
        d_field = torch.from_numpy(field.reshape(-1)).cuda()
        bricks = torch.zeros(rafi.c2_bricks_floats(n, brick), dtype=torch.float32, device="cuda")
        rafi.rf_c2_make_bricks(d_field, n, brick, bricks, s)
        del d_field
        d_seeds = torch.from_numpy(inputs.c2_seeds(count, n, seed=2)).cuda()
        d_sets = torch.zeros(count, dtype=torch.int32, device="cuda")
        res = torch.zeros((count, 8), dtype=torch.int32, device="cuda")
        with rafi.Context(R, 32, count) as ctx:
            e0.record(s)
            _, rounds, fwd = rafi.rf_c2_run(ctx.handle, bricks, d_seeds, d_sets, count, n, brick, 0.25, 2000, 0,
                                            res, 0, stream=s)
            e1.record(s)
            torch.cuda.synchronize()
        steps = int(res[:, 4].cpu().numpy().view(np.uint32).astype(np.int64).sum())
        out.update(workload=f"512^3 curl-noise field, 4x4x4 ranks, {count} seeds, until brick exit, host loop",
                   ms=e0.elapsed_time(e1), rounds=rounds, particle_steps=steps,
                   particle_steps_per_s=steps / (e0.elapsed_time(e1) * 1e-3))
    elif args.section == "c3":
        n, brick, w, h, spp = 256, 128, 512, 512, 4
        vol = inputs.c0_volume(n)
        cam = inputs.c0_camera(n, w, h)
        dv = torch.from_numpy(vol.reshape(-1)).cuda()
        bricks = torch.zeros(rafi.c0_bricks_floats(n, brick), dtype=torch.float32, device="cuda")
        rafi.rf_c0_make_bricks(dv, n, brick, bricks, s)
        nr = w * h * spp
        rayC = torch.zeros(nr, dtype=torch.float32, device="cuda")
        rayClo = torch.zeros(nr, dtype=torch.float32, device="cuda")
        img = torch.zeros(w * h, dtype=torch.float32, device="cuda")
        gimg = torch.ones(w * h, dtype=torch.float32, device="cuda")
        grad = torch.zeros(n ** 3, dtype=torch.float32, device="cuda")
        out["workload"] = "256^3 blob density, 2x2x2 ranks, 512x512 at 4 spp (compensated colour sums)"
        with rafi.Context(8, 64, nr) as ctx:
            for name, fn in (("forward", lambda: rafi.rf_c3_render(ctx.handle, bricks, cam, n, brick, w, h, spp, 3,
                                                                    rayC, img, stream=s, ray_c_lo=rayClo)),
                             ("adjoint", lambda: rafi.rf_c3_adjoint(ctx.handle, bricks, cam, n, brick, w, h, spp, 3,
                                                                     rayC, gimg, grad, stream=s, ray_c_lo=rayClo))):
                e0.record(s)
                fn()
                e1.record(s)
                torch.cuda.synchronize()
                out[name] = {"ms": e0.elapsed_time(e1), "rays_per_s": nr / (e0.elapsed_time(e1) * 1e-3)}
    else:
        n, brick, spp = 512, 128, 16
        R = (n // brick) ** 3
        vol, smax = inputs.c4_volume(n)
        views = inputs.c4_views(n, sizes=((512, 512),))
        bricks = torch.zeros(rafi.c0_bricks_floats(n, brick), dtype=torch.float32, device="cuda")
        dv = torch.from_numpy(vol.reshape(-1)).cuda()
        rafi.rf_c0_make_bricks(dv, n, brick, bricks, s)
        del dv
        paths = 512 * 512 * spp
        score = torch.zeros(512 * 512, dtype=torch.float32, device="cuda")
        with rafi.Context(R, 64, paths) as ctx:
            e0.record(s)
            rounds, fwd = rafi.rf_c4_render(ctx.handle, bricks, n, brick, smax, views, spp, 4, score, 0, stream=s)
            e1.record(s)
            torch.cuda.synchronize()
        out.update(workload="512^3 noise (mean optical depth 8), 4x4x4 ranks, one 512x512 view at 16 spp, host loop",
                   ms=e0.elapsed_time(e1), rounds=rounds, paths_per_s=paths / (e0.elapsed_time(e1) * 1e-3))
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--items", type=int, default=N_ITEMS)
    ap.add_argument("--skip-extra", action="store_true",
                    help="leave out the streamline, differentiable and transport workloads")
    ap.add_argument("--section", choices=["c0", "c1", "c2", "c3", "c4"], default=None,
                    help="run one workload alone at a profiling size and print its own JSON line (c1: one "
                         "persistent-kernel launch of the microbenchmark at --items; c2-c4: a host loop)")
    ap.add_argument("--law", type=int, default=0, choices=list(MODES), help="destination law of --section c1")
    ap.add_argument("--joint", action="store_true", help="--section c1: the three laws in one launch")
    ap.add_argument("--round-log", default=None, help="--section c1: write the kernel's round log to this JSON file")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.section:
        return run_section(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
