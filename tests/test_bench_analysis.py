"""The bench's own arithmetic, on CPU: the per-round rates it derives from the
persistent kernel's round log, and the gate that reports measured DRAM
traffic only for the sources it was captured from."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _log():
    # rounds: {t_start, t_count_end, t_barrier1, t_scatter_end, t_barrier2, n_in, n_next} in ns
    rows, t = [], 1000
    sizes = [(1 << 22, 3774874), (3774874, 3397386), (3397386, 1 << 19), (1 << 19, 300), (300, 0)]
    for n_in, n_next in sizes:
        big = n_in >= (1 << 20)
        d = [10_000, 2_000, 300_000 if big else 5_000, 3_000] if n_in > 512 else [1_500, 0, 400, 0]
        c = np.cumsum([t] + d)
        rows.append([int(c[0]), int(c[1]), int(c[2]), int(c[3]), int(c[4]), n_in, n_next])
        t = int(c[4]) + 100
    return rows


def test_phase_rates_follow_the_forwarding_bytes():
    rows = _log()
    r = bench.phase_rates(rows, 64)
    lg = np.array(rows, dtype=np.float64)
    big = lg[:, 5] >= (1 << 20)
    assert r["rounds"] == 5 and r["rounds_ge_2^20"] == 3
    # 2 x 64 B per forwarded item (the round's n_next) over whole rounds, start to second barrier
    want = (lg[big, 6] * 128).sum() / ((lg[big, 4] - lg[big, 0]).sum() * 1e-9) / 1e9
    assert r["fwd_gbs_ge_2^20"] == pytest.approx(want)
    # the scatter phase moves every queued item (read + write) and 4 B destinations
    scat = (lg[big, 5] * 132 + lg[big, 6] * 4).sum() / ((lg[big, 4] - lg[big, 2]).sum() * 1e-9) / 1e9
    assert r["scatter_gbs_ge_2^20"] == pytest.approx(scat)
    # size classes: one round on one CTA (at most 512 items), one on the grid below 2^20
    assert r["rounds_solo_le_512"] == 1 and r["rounds_grid_lt_2^20"] == 1
    assert r["us_per_round_solo_le_512"] == pytest.approx(1.9)
    assert r["us_split_grid_lt_2^20"] == pytest.approx([10.0, 2.0, 5.0, 3.0])
    assert r["round_ms_total"] == pytest.approx((rows[-1][4] - rows[0][0]) * 1e-6)


def test_traffic_is_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    doc = {"code_sha256": bench.rounds_kernel_code_hash(), "bytes_per_full_size_launch": 123.0}
    (prof / "rounds_kernel_traffic.json").write_text(json.dumps(doc))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the hash is taken over the package's sources, which the temporary root lacks: link them
    os.symlink(os.path.join(ROOT, "paper_2605_30294_gb300"), tmp_path / "paper_2605_30294_gb300")
    assert bench.rounds_kernel_traffic() == 123.0
    doc["code_sha256"] = "0" * 64
    (prof / "rounds_kernel_traffic.json").write_text(json.dumps(doc))
    assert bench.rounds_kernel_traffic() is None

