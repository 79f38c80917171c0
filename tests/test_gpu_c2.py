"""GPU parity: streamlines through a brick-partitioned field (Sec. 5.4) vs the oracle.

The oracle integrates every particle through the unpartitioned field; the GPU
forwards it between the ranks that own the bricks it crosses.  RK4 and the
trilinear taps run in the same float order on both sides (no contraction), so
final positions, step counts, stop reasons and hop counts agree exactly; the
stated tolerance for positions is a max relative error of 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_30294_gb300 import inputs, rafi

from gpu_util import dev, stream, to_dev

pytestmark = pytest.mark.gpu

_FIELDS = {}


def field(n):
    if n not in _FIELDS:
        _FIELDS[n] = inputs.c2_field(n)[0]
    return _FIELDS[n]


def run_gpu(f, n, brick, seeds, set_ids=None, h=0.25, max_steps=2000, spr=0, batched=False, shape=0):
    R = (n // brick) ** 3
    s = stream()
    bricks = torch.zeros(rafi.c2_bricks_floats(n, brick), dtype=torch.float32, device=dev())
    rafi.rf_c2_make_bricks(to_dev(f.reshape(-1)), n, brick, bricks, s)
    cnt = len(seeds)
    out = torch.zeros((cnt, 8), dtype=torch.int32, device=dev())
    sid = to_dev(np.asarray(set_ids, np.uint32)) if set_ids is not None else None
    with rafi.Context(R, 32, cnt) as ctx:
        rafi.rf_set_batched_config(ctx.handle, rafi.RF_POLICY_STREAMLINES, rafi.RF_FORM_PERSISTENT, shape)
        st, rounds, fwd = rafi.rf_c2_run(ctx.handle, bricks, to_dev(seeds), sid, cnt, n, brick, h, max_steps, spr,
                                         out, batched, stream=s)
    o = out.cpu().numpy().view(np.uint32)
    return dict(pos=o[:, :3].copy().view(np.float32), id=o[:, 3], steps=o[:, 4], hops=o[:, 5], set=o[:, 6],
                status=o[:, 7], rounds=rounds, forwarded=fwd)


def check_against_oracle(got, want, idx=None):
    if idx is None:
        idx = np.arange(len(want["steps"]))
    np.testing.assert_array_equal(got["status"][idx], want["status"])
    np.testing.assert_array_equal(got["steps"][idx], want["steps"])
    np.testing.assert_array_equal(got["hops"][idx], want["hops"])
    rel = np.abs(got["pos"][idx] - want["pos"]) / np.maximum(np.abs(want["pos"]), 1.0)
    assert rel.max() <= 1e-5, rel.max()


@pytest.mark.parametrize("batched", [0, 1, 2], ids=["host_loop", "persistent", "graph"])
@pytest.mark.parametrize("spr", [0, 1])
def test_streamlines_match_oracle(batched, spr):
    n, brick = 64, 16
    f = field(n)
    seeds = inputs.c2_seeds(3000, n, seed=5)
    max_steps = 600 if spr else 2000
    got = run_gpu(f, n, brick, seeds, max_steps=max_steps, spr=spr, batched=batched)
    want = oracle.c2_trace(f, seeds, brick, 0.25, max_steps)
    np.testing.assert_array_equal(got["id"], np.arange(len(seeds)))
    check_against_oracle(got, want)
    assert set(np.unique(got["status"])) <= {1, 2, 3}
    if spr == 0:
        # only brick changes forward a particle
        assert got["forwarded"] == int(want["hops"].sum())
    else:
        # every step forwards the particle (to itself or a neighbour) except one that
        # leaves the grid, and the last step of a particle that hits the step cap
        # forwards it only when it enters another brick
        total = int(want["steps"].sum()) - int((want["status"] == oracle.EXITED).sum())
        capped = int((want["status"] == oracle.MAXSTEPS).sum())
        assert total - capped <= got["forwarded"] <= total


def test_partition_independence():
    n = 64
    f = field(n)
    seeds = inputs.c2_seeds(2000, n, seed=6)
    runs = [run_gpu(f, n, b, seeds, batched=True) for b in (64, 32, 16)]
    for r in runs[1:]:
        np.testing.assert_array_equal(r["pos"].view(np.uint32), runs[0]["pos"].view(np.uint32))
        np.testing.assert_array_equal(r["steps"], runs[0]["steps"])
        np.testing.assert_array_equal(r["status"], runs[0]["status"])
    assert runs[0]["hops"].max() == 0 and runs[2]["hops"].sum() > runs[1]["hops"].sum() > 0


def test_uneven_seed_sets_in_one_launch():
    n, brick = 64, 16
    f = field(n)
    sizes = [max(1, s // 256) for s in inputs.c2_seed_set_sizes()]
    seeds = inputs.c2_seeds(sum(sizes), n, seed=7)
    set_ids = np.repeat(np.arange(len(sizes), dtype=np.uint32), sizes)
    got = run_gpu(f, n, brick, seeds, set_ids=set_ids, batched=True)
    np.testing.assert_array_equal(got["set"], set_ids)
    want = oracle.c2_trace(f, seeds, brick, 0.25, 2000)
    check_against_oracle(got, want)
    for form in (0, 2):  # the host loop and the graph loop give the same particles
        other = run_gpu(f, n, brick, seeds, set_ids=set_ids, batched=form)
        np.testing.assert_array_equal(other["pos"].view(np.uint32), got["pos"].view(np.uint32))
        np.testing.assert_array_equal(other["steps"], got["steps"])
        assert other["forwarded"] == got["forwarded"] and other["rounds"] == got["rounds"]


def test_full_size_sampled():
    # 512^3 field, 4x4x4 ranks of 128^3 bricks, 2^22 seeds: the configured workload
    n, brick, count = 512, 128, 1 << 22
    f = field(n)
    seeds = inputs.c2_seeds(count, n, seed=2)
    got = run_gpu(f, n, brick, seeds, batched=True)
    np.testing.assert_array_equal(got["id"], np.arange(count))
    assert set(np.unique(got["status"])) <= {1, 2, 3}
    assert got["forwarded"] == int(got["hops"].astype(np.int64).sum())
    sample = np.random.default_rng(1).choice(count, size=256, replace=False)
    want = oracle.c2_trace(f, seeds[sample], brick, 0.25, 2000)
    check_against_oracle(got, want, idx=sample)


@pytest.mark.parametrize("shape", range(len(rafi.rf_rounds_shapes(rafi.RF_POLICY_STREAMLINES))))
@pytest.mark.parametrize("spr", [0, 1])
def test_every_persistent_shape_matches_oracle(shape, spr):
    # each shape the autotuner may pick (threads, tile, CTAs per SM) gives the
    # oracle's particles exactly; RF_FORM_TUNED runs the form set on the context
    n, brick = 64, 16
    f = field(n)
    seeds = inputs.c2_seeds(3000, n, seed=6)
    max_steps = 600 if spr else 2000
    want = oracle.c2_trace(f, seeds, brick, 0.25, max_steps)
    got = run_gpu(f, n, brick, seeds, max_steps=max_steps, spr=spr, batched=rafi.RF_FORM_TUNED, shape=shape)
    check_against_oracle(got, want)
