"""GPU parity: several microbenchmark runs in one persistent launch.

rf_c1_run_batched_runs carries independent runs (each with its own items and
destination law) through the same rounds: the ranks' queues hold every run's
items, each run retires into a sink of its own.  A stable partition of the
joint queue, restricted to one run, is that run's own stable partition
(Sec. 4.2.1), so each run's retirement buffer must equal the oracle's
round-by-round simulation of that run alone, row for row and word for word,
and its round count the oracle's.  The checks cover several sizes (rounds
above and below 2^20 items, the one-CTA tail), every law order and run count,
every compiled shape, page-locked host buffers, the full benched size (three
runs of 2^24 items), and the argument checks.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_30294_gb300 import inputs, rafi

from gpu_util import dev, stream, to_dev

pytestmark = pytest.mark.gpu

R = 64
GRID = (4, 4, 4)
U, Z, T = rafi.RF_C1_UNIFORM, rafi.RF_C1_ZIPF, rafi.RF_C1_NBR6


def _items(n, seeds):
    return np.concatenate([inputs.c1_items(n, seed=s) for s in seeds]) if n else np.zeros((0, 16), np.uint32)


def _runs(items, n, seed, modes, ctx=None, host=False, round_log=None):
    """One call; returns (per-run retired rows, counts, rounds, forwarded).  host:
    False (device buffers), True (page-locked host buffers: runs launched one by
    one, copies overlapped) or "pageable" (plain host memory: one joint launch)."""
    k = len(modes)
    s = stream()
    own = ctx is None
    ctx = ctx or rafi.Context(R, 64, max(k * n, 1))
    try:
        if host == "pageable":
            h_items = np.ascontiguousarray(items).reshape(-1, 16)
            h_ret = np.zeros((max(k * n, 1), 16), np.uint32)
            st, cnt, rounds, fwd = rafi.rf_c1_run_batched_runs(ctx.handle, h_items, n, seed, modes, 1.1, GRID,
                                                               h_ret, host_memory=True, stream=s)
            got = h_ret
        elif host:
            h_items = torch.from_numpy(np.ascontiguousarray(items).view(np.int32).reshape(-1, 16)).pin_memory()
            h_ret = torch.zeros((max(k * n, 1), 16), dtype=torch.int32).pin_memory()
            st, cnt, rounds, fwd = rafi.rf_c1_run_batched_runs(ctx.handle, h_items.data_ptr(), n, seed, modes, 1.1,
                                                               GRID, h_ret.data_ptr(), host_memory=True, stream=s)
            got = h_ret.numpy().view(np.uint32)
        else:
            ret = torch.full((max(k * n, 1), 16), -1, dtype=torch.int32, device=dev())
            d_items = to_dev(items) if k * n else torch.zeros((1, 16), dtype=torch.int32, device=dev())
            st, cnt, rounds, fwd = rafi.rf_c1_run_batched_runs(ctx.handle, d_items, n, seed, modes, 1.1, GRID, ret,
                                                               stream=s, round_log=round_log,
                                                               round_log_cap=0 if round_log is None else
                                                               len(round_log) // 7)
            got = ret.cpu().numpy().view(np.uint32)
        assert st == rafi.RF_OK
        return [got[j * n:(j + 1) * n] for j in range(k)], cnt, rounds, fwd
    finally:
        if own:
            ctx.close()


def _check_against_oracle(items, n, seed, modes, got, cnt, rounds, fwd):
    total_fwd = 0
    for j, mode in enumerate(modes):
        want = oracle.c1_rounds(items[j * n:(j + 1) * n], R, seed, mode, grid=GRID)
        assert cnt[j] == n, f"run {j}: {cnt[j]} of {n} retired"
        assert rounds[j] == int(want["rounds"]), f"run {j}"
        bad = np.flatnonzero(np.any(got[j] != want["retired_items"], axis=1))
        assert bad.size == 0, f"run {j} (law {mode}): {bad.size} rows differ, first at {bad[:4]}"
        total_fwd += int(want["active"][1:].sum())
    assert fwd == total_fwd


@pytest.mark.parametrize("n", [1, 777, 20011, 300007, 1 << 20])
def test_three_laws_each_retire_in_the_oracle_order(n):
    seed, modes = 51, [U, Z, T]
    items = _items(n, (5, 6, 7))
    got, cnt, rounds, fwd = _runs(items, n, seed, modes)
    _check_against_oracle(items, n, seed, modes, got, cnt, rounds, fwd)


@pytest.mark.parametrize("modes", [[T], [Z, U], [T, T], [Z, T, U], [U, Z, T, Z]], ids=str)
def test_any_run_count_and_law_order(modes):
    n, seed = 50021, 53
    items = _items(n, range(11, 11 + len(modes)))
    got, cnt, rounds, fwd = _runs(items, n, seed, modes)
    _check_against_oracle(items, n, seed, modes, got, cnt, rounds, fwd)


def test_same_items_in_every_run_as_the_bench_runs_them():
    # the bench gives the three runs the same seeded items: every run then
    # retires each item in the same round (the retire draw ignores the law)
    n, seed, modes = 100003, 1, [U, Z, T]
    one = inputs.c1_items(n, seed=1)
    items = np.concatenate([one] * 3)
    got, cnt, rounds, fwd = _runs(items, n, seed, modes)
    _check_against_oracle(items, n, seed, modes, got, cnt, rounds, fwd)
    assert rounds[0] == rounds[1] == rounds[2]


@pytest.mark.parametrize("shape", range(len(rafi.rf_rounds_shapes(rafi.RF_POLICY_MICROBENCH))))
def test_every_persistent_shape(shape):
    n, seed, modes = 20011, 57, [Z, T, U]
    items = _items(n, (21, 22, 23))
    with rafi.Context(R, 64, 3 * n) as ctx:
        rafi.rf_set_batched_config(ctx.handle, rafi.RF_POLICY_MICROBENCH, rafi.RF_FORM_PERSISTENT, shape)
        got, cnt, rounds, fwd = _runs(items, n, seed, modes, ctx=ctx)
    _check_against_oracle(items, n, seed, modes, got, cnt, rounds, fwd)


def test_joint_launch_equals_separate_launches_and_host_buffers():
    # the same runs launched one by one (rf_c1_run_batched), jointly from
    # device buffers, from page-locked host buffers (one launch per run, copies
    # overlapped) and from pageable host buffers (joint launch, staged sink):
    # identical retirement buffers, rounds and forwards
    n, seed, modes = 300007, 59, [T, U, Z]
    items = _items(n, (31, 32, 33))
    s = stream()
    sep, sep_rounds, sep_fwd = [], [], 0
    with rafi.Context(R, 64, 3 * n) as ctx:
        for j, mode in enumerate(modes):
            ret = torch.zeros((n, 16), dtype=torch.int32, device=dev())
            st, cnt, rounds, fwd = rafi.rf_c1_run_batched(ctx.handle, to_dev(items[j * n:(j + 1) * n]), n, seed,
                                                          mode, 1.1, GRID, ret, stream=s)
            assert st == rafi.RF_OK and cnt == n
            sep.append(ret.cpu().numpy().view(np.uint32))
            sep_rounds.append(rounds)
            sep_fwd += fwd
        for host in (False, True, "pageable"):
            got, cnt, rounds, fwd = _runs(items, n, seed, modes, ctx=ctx, host=host)
            assert cnt == [n] * 3 and rounds == sep_rounds and fwd == sep_fwd
            for j in range(3):
                np.testing.assert_array_equal(got[j], sep[j])


def test_round_log_covers_the_joint_rounds():
    n, seed, modes = 1 << 18, 61, [U, Z, T]
    items = _items(n, (41, 42, 43))
    log = torch.zeros(7 * 512, dtype=torch.int64, device=dev())
    got, cnt, rounds, fwd = _runs(items, n, seed, modes, round_log=log)
    lg = log.cpu().numpy().reshape(-1, 7)
    lg = lg[lg[:, 0] > 0]
    assert len(lg) == max(rounds)
    assert lg[0, 5] == 3 * n  # round 0 holds every run's items
    assert int(lg[:, 6].sum()) == fwd
    assert np.all(lg[1:, 5] == lg[:-1, 6])  # each round delivers the next one's queue
    assert np.all(np.diff(lg[:, 0]) >= 0)


@pytest.mark.parametrize("mode_set", [[U, Z, T]])
def test_full_size_three_runs_every_word_matches_oracle(mode_set):
    # The benched configuration: three runs of 2^24 x 64 B items (the same
    # seeded items, laws uniform, Zipf 1.1 and 6-neighbour torus) over 64 ranks
    # in one launch.  Every run's retirement buffer equals the oracle's
    # round-by-round simulation of that run, row for row, all 16 words.
    n, seed = 1 << 24, 1
    one = inputs.c1_items(n, seed=1)
    s = stream()
    d_one = to_dev(one)
    d_items = torch.cat([d_one, d_one, d_one])
    del d_one
    with rafi.Context(R, 64, 3 * n) as ctx:
        ret = torch.full((3 * n, 16), -1, dtype=torch.int32, device=dev())
        st, cnt, rounds, fwd = rafi.rf_c1_run_batched_runs(ctx.handle, d_items, n, seed, mode_set, 1.1, GRID, ret,
                                                           stream=s)
        assert st == rafi.RF_OK and cnt == [n] * 3
        total_fwd = 0
        for j, mode in enumerate(mode_set):
            want = oracle.c1_rounds(one, R, seed, mode, grid=GRID)
            assert rounds[j] == int(want["rounds"])
            total_fwd += int(want["active"][1:].sum())
            got = ret[j * n:(j + 1) * n].cpu().numpy().view(np.uint32)
            bad = np.flatnonzero(np.any(got != want["retired_items"], axis=1))
            assert bad.size == 0, f"run {j}: {bad.size} rows differ, first at {bad[:4]}"
            del want, got
        assert fwd == total_fwd
    del d_items, ret
    torch.cuda.empty_cache()


def test_argument_checks():
    n = 1000
    items = torch.zeros((4 * n, 16), dtype=torch.int32, device=dev())
    ret = torch.zeros((4 * n, 16), dtype=torch.int32, device=dev())
    s = stream()
    with rafi.Context(R, 64, 3 * n) as ctx:
        for modes in ([], [U] * 5, [U, 7]):
            with pytest.raises(rafi.RafiError) as e:
                rafi.rf_c1_run_batched_runs(ctx.handle, items, n, 1, modes, 1.1, GRID, ret, stream=s)
            assert e.value.status == rafi.RF_ERR_ARG
        with pytest.raises(rafi.RafiError) as e:  # four runs of n do not fit a capacity of 3 n
            rafi.rf_c1_run_batched_runs(ctx.handle, items, n, 1, [U] * 4, 1.1, GRID, ret, stream=s)
        assert e.value.status == rafi.RF_ERR_ARG and "capacity" in rafi.rf_last_error()
        with pytest.raises(rafi.RafiError) as e:  # a torus that does not have 64 ranks
            rafi.rf_c1_run_batched_runs(ctx.handle, items, n, 1, [U, T], 1.1, (4, 4, 2), ret, stream=s)
        assert e.value.status == rafi.RF_ERR_ARG
        # the context still runs
        got, cnt, rounds, fwd = _runs(_items(n, (1, 2)), n, 3, [Z, T], ctx=ctx)
        assert cnt == [n, n]
