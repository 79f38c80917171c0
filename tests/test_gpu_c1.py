"""GPU parity: the forwarding microbenchmark against the oracle.

Small runs compare the whole final payload multiset bit-exactly, the round
count, the forward count and the per-round queues (bit-exact in the
deterministic mode, whose queue order equals the oracle's; after a canonical
sort per rank segment in the atomic-append mode).  The full-size run
(2^24 x 64 B items over 64 ranks, as timed by bench.py) is checked on sampled
items the oracle walks one by one, plus invariants that hold at any size.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_30294_gb300 import inputs, rafi

from gpu_util import canonical_rows, dev, stream, to_dev

pytestmark = pytest.mark.gpu

R = 64
GRID = (4, 4, 4)
MODES = [rafi.RF_C1_UNIFORM, rafi.RF_C1_ZIPF, rafi.RF_C1_NBR6]


def _run(items, seed, mode, deterministic=False, host=False):
    n = len(items)
    s = stream()
    with rafi.Context(R, 64, n) as ctx:
        if host:
            retired = np.zeros((n, 16), np.uint32)
            st, cnt, rounds, fwd = rafi.rf_c1_run(ctx.handle, items.ctypes.data, n, seed, mode, 1.1, GRID,
                                                  retired.ctypes.data, deterministic, True, stream=s)
            return retired[:cnt], rounds, fwd
        d_items = to_dev(items)
        retired = torch.zeros((n, 16), dtype=torch.int32, device=dev())
        st, cnt, rounds, fwd = rafi.rf_c1_run(ctx.handle, d_items, n, seed, mode, 1.1, GRID, retired,
                                              deterministic, False, stream=s)
        return retired[:cnt].cpu().numpy().view(np.uint32), rounds, fwd


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("deterministic", [False, True])
def test_run_matches_oracle_multiset(mode, deterministic):
    n, seed = 20011, 3
    items = inputs.c1_items(n, seed=seed)
    got, rounds, fwd = _run(items, seed, mode, deterministic)
    final, hops, _, _ = oracle.c1_walk(items, R, seed, mode, grid=GRID)
    assert len(got) == n
    assert rounds == int(hops.max()) + 1
    assert fwd == int(hops.sum())
    np.testing.assert_array_equal(canonical_rows(got), canonical_rows(final))


def test_host_memory_run_matches_device_run():
    n, seed = 10000, 4
    items = inputs.c1_items(n, seed=seed)
    a, ra, fa = _run(items, seed, rafi.RF_C1_ZIPF)
    b, rb, fb = _run(items, seed, rafi.RF_C1_ZIPF, host=True)
    assert (ra, fa) == (rb, fb)
    np.testing.assert_array_equal(canonical_rows(a), canonical_rows(b))


def _queue(ctx, n, s):
    q = torch.zeros((max(n, 1), 16), dtype=torch.int32, device=dev())
    off = torch.zeros(R + 1, dtype=torch.int32, device=dev())
    rafi.rf_snapshot(ctx.handle, q, off, s)
    torch.cuda.synchronize()
    o = off.cpu().numpy().astype(np.int64)
    return q.cpu().numpy().view(np.uint32)[: o[-1]], o


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("deterministic", [True, False])
def test_round_queues_match_oracle(mode, deterministic):
    n, seed, rounds_checked = 6000, 7, 5
    items = inputs.c1_items(n, seed=seed)
    s = stream()
    with rafi.Context(R, 64, n) as ctx:
        retired = torch.zeros((n, 16), dtype=torch.int32, device=dev())
        rcount = torch.zeros(1, dtype=torch.int64, device=dev())
        rafi.rf_c1_seed(ctx.handle, to_dev(items), n, s)
        st, active = rafi.rf_exchange(ctx.handle, s)
        for k in range(rounds_checked):
            want = oracle.c1_rounds(items, R, seed, mode, grid=GRID, dump_round=k)
            q, off = _queue(ctx, active, s)
            np.testing.assert_array_equal(off.astype(np.uint64), want["dump_offsets"])
            assert active == int(want["active"][k])
            if deterministic:
                np.testing.assert_array_equal(q, want["dump_items"])
            else:
                for r in range(R):
                    np.testing.assert_array_equal(canonical_rows(q[off[r]:off[r + 1]]),
                                                  canonical_rows(want["dump_items"][off[r]:off[r + 1]]))
            before = int(rcount.item())
            rafi.rf_c1_work(ctx.handle, seed, k, mode, 1.1, GRID, retired, rcount, n, deterministic, s)
            st, nxt = rafi.rf_exchange(ctx.handle, s)
            # conservation: active_k = retired_k + active_{k+1}
            assert active == (int(rcount.item()) - before) + nxt
            assert int(rcount.item()) - before == int(want["retired"][k])
            stats = rafi.rf_stats(ctx.handle)
            assert stats.holes == (active - nxt if deterministic else 0)
            active = nxt


def test_full_size_sampled_parity():
    # the bench workload: 2^24 items x 64 B, 64 ranks, each destination law
    n, seed = 1 << 24, 1
    items = _full_items()
    d_items = to_dev(items)
    s = stream()
    rng = np.random.default_rng(0)
    sample = rng.choice(n, size=4096, replace=False)
    key_in = (items[:, 0].astype(np.uint64) << np.uint64(32)) | items[:, 1].astype(np.uint64)
    assert len(np.unique(key_in)) == n  # (w0, w1) identifies an item
    with rafi.Context(R, 64, n) as ctx:
        retired = torch.zeros((n, 16), dtype=torch.int32, device=dev())
        for mode in MODES:
            st, cnt, rounds, fwd = rafi.rf_c1_run(ctx.handle, d_items, n, seed, mode, 1.1, GRID, retired,
                                                  stream=s)
            got = retired.cpu().numpy().view(np.uint32)
            assert cnt == n
            key = (got[:, 0].astype(np.uint64) << np.uint64(32)) | got[:, 1].astype(np.uint64)
            order = np.argsort(key)
            # invariants at full size: words 0..12 are the input's, hop counts add up
            np.testing.assert_array_equal(key[order], np.sort(key_in))
            inv = np.argsort(key_in)
            np.testing.assert_array_equal(got[order, :13], items[inv, :13])
            assert int((got[order, 15] - items[inv, 15]).astype(np.int64).sum()) == fwd
            assert 9 * n * 0.99 < fwd < 9 * n * 1.01
            # sampled items walked one by one by the oracle, each from its own start rank
            final, _, _, _ = oracle.c1_walk(items[sample], R, seed, mode, grid=GRID,
                                            start_ranks=(sample % R).astype(np.int32))
            pos = np.searchsorted(key[order], key_in[sample])
            mism = int(np.sum(np.any(got[order[pos]] != final, axis=1)))
            assert mism == 0


def test_max_rounds_guard():
    n, seed = 5000, 2
    items = inputs.c1_items(n, seed=seed)
    s = stream()
    with rafi.Context(R, 64, n) as ctx:
        retired = torch.zeros((n, 16), dtype=torch.int32, device=dev())
        st, cnt, rounds, fwd = rafi.rf_c1_run(ctx.handle, to_dev(items), n, seed, rafi.RF_C1_UNIFORM, 1.1, GRID,
                                              retired, max_rounds=3, stream=s,
                                              allow=(rafi.RF_ERR_MAX_ROUNDS,))
        assert st == rafi.RF_ERR_MAX_ROUNDS and rounds == 3 and cnt < n


# ---------------------------------------------------------------------------
# batched form: all rounds in one persistent kernel
# ---------------------------------------------------------------------------
def _run_batched(items, seed, mode, host=False, max_rounds=100000, ctx=None, allow=(), fuse=True):
    n = len(items)
    s = stream()
    own = ctx is None
    ctx = ctx or rafi.Context(R, 64, n)
    try:
        if host:
            retired = np.zeros((n, 16), np.uint32)
            st, cnt, rounds, fwd = rafi.rf_c1_run_batched(ctx.handle, items.ctypes.data, n, seed, mode, 1.1, GRID,
                                                          retired.ctypes.data, True, max_rounds, s, allow=allow,
                                                          step_on_arrival=fuse)
            return retired[:cnt], rounds, fwd, st
        retired = torch.zeros((n, 16), dtype=torch.int32, device=dev())
        st, cnt, rounds, fwd = rafi.rf_c1_run_batched(ctx.handle, to_dev(items), n, seed, mode, 1.1, GRID, retired,
                                                      False, max_rounds, s, allow=allow, step_on_arrival=fuse)
        return retired[:cnt].cpu().numpy().view(np.uint32), rounds, fwd, st
    finally:
        if own:
            ctx.close()


@pytest.mark.parametrize("fuse", [True, False], ids=["step_on_arrival", "step_in_place"])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [1, 777, 20011, 300007])
def test_batched_matches_oracle_multiset(mode, n, fuse):
    seed = 5
    items = inputs.c1_items(n, seed=seed)
    got, rounds, fwd, st = _run_batched(items, seed, mode, fuse=fuse)
    final, hops, _, _ = oracle.c1_walk(items, R, seed, mode, grid=GRID)
    assert st == rafi.RF_OK and len(got) == n
    assert rounds == int(hops.max()) + 1
    assert fwd == int(hops.sum())
    np.testing.assert_array_equal(canonical_rows(got), canonical_rows(final))


@pytest.mark.parametrize("fuse", [True, False], ids=["step_on_arrival", "step_in_place"])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,stops", [(50000, (0, 1, 2, 3, 7, 8)), (2000, (9, 15, 16, 30, 45))],
                         ids=["grid_rounds", "one_cta_tail"])
def test_batched_round_queues_bit_exact(mode, fuse, n, stops):
    # stopping after k rounds leaves round k's incoming queue, in the serial order
    # (with steps on arrival: whether the last fused scatter lands in either
    # queue, and, for the small run, after rounds kept in one CTA's shared memory)
    seed = 8
    items = inputs.c1_items(n, seed=seed)
    s = stream()
    for k in stops:
        want = oracle.c1_rounds(items, R, seed, mode, grid=GRID, dump_round=k)
        with rafi.Context(R, 64, n) as ctx:
            got, rounds, fwd, st = _run_batched(items, seed, mode, max_rounds=k, ctx=ctx,
                                                allow=(rafi.RF_ERR_MAX_ROUNDS,), fuse=fuse)
            assert rounds == k
            assert fwd == int(want["active"][1:k + 1].sum())
            assert rafi.rf_num_active(ctx.handle) == int(want["active"][k])
            q, off = _queue(ctx, n, s)
        np.testing.assert_array_equal(off.astype(np.uint64), want["dump_offsets"])
        np.testing.assert_array_equal(q, want["dump_items"])
        # the retired items so far are the oracle's first k rounds of retirements,
        # in its order (round by round, queue order within a round)
        ret = int(want["retired"][:k].sum())
        assert len(got) == ret
        np.testing.assert_array_equal(got, want["retired_items"][:ret])


def test_batched_host_memory_and_round_log():
    n, seed = 100000, 9
    items = inputs.c1_items(n, seed=seed)
    a, ra, fa, _ = _run_batched(items, seed, rafi.RF_C1_NBR6)
    b, rb, fb, _ = _run_batched(items, seed, rafi.RF_C1_NBR6, host=True)
    assert (ra, fa) == (rb, fb)
    np.testing.assert_array_equal(canonical_rows(a), canonical_rows(b))
    s = stream()
    log = torch.zeros(7 * 512, dtype=torch.int64, device=dev())
    retired = torch.zeros((n, 16), dtype=torch.int32, device=dev())
    with rafi.Context(R, 64, n) as ctx:
        st, cnt, rounds, fwd = rafi.rf_c1_run_batched(ctx.handle, to_dev(items), n, seed, rafi.RF_C1_NBR6, 1.1,
                                                      GRID, retired, False, 100000, s, log, 512)
    lg = log.cpu().numpy().reshape(-1, 7)[:rounds]
    t = lg[:, :5]
    assert rounds == ra and np.all(t > 0)
    assert np.all(np.diff(t, axis=1) >= 0) and np.all(t[1:, 0] >= t[:-1, 4])
    # counts: n_in of round k+1 = n_next of round k; round 0 starts with all items
    assert lg[0, 5] == n and np.all(lg[1:, 5] == lg[:-1, 6]) and lg[-1, 6] == 0
    assert int(lg[:, 6].sum()) == fwd


@pytest.mark.parametrize("fuse", [True, False], ids=["step_on_arrival", "step_in_place"])
def test_batched_pinned_host_buffers(fuse):
    # page-locked host buffers: the kernel writes the retired items straight
    # into the host buffer; the result equals the device-memory run's
    n, seed = 200003, 12
    items = inputs.c1_items(n, seed=seed)
    s = stream()
    h_items = torch.from_numpy(items.view(np.int32)).pin_memory()
    h_ret = torch.zeros((n, 16), dtype=torch.int32).pin_memory()
    d_ret = torch.zeros((n, 16), dtype=torch.int32, device=dev())
    with rafi.Context(R, 64, n) as ctx:
        for mode in MODES:
            h_ret.zero_()
            st, ch, rh, fh = rafi.rf_c1_run_batched(ctx.handle, h_items.data_ptr(), n, seed, mode, 1.1, GRID,
                                                    h_ret.data_ptr(), True, stream=s, step_on_arrival=fuse)
            st, cd, rd, fd = rafi.rf_c1_run_batched(ctx.handle, to_dev(items), n, seed, mode, 1.1, GRID, d_ret,
                                                    False, stream=s, step_on_arrival=fuse)
            assert (ch, rh, fh) == (cd, rd, fd) and ch == n
            np.testing.assert_array_equal(h_ret.numpy(), d_ret.cpu().numpy())


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("deterministic", [True, False])
def test_graph_form(mode, deterministic):
    # the host loop's rounds inside a CUDA graph: same rounds and forwards, the
    # oracle's final payloads; stopping after k rounds leaves round k's queue
    n, seed = 20011, 13
    items = inputs.c1_items(n, seed=seed)
    final, hops, _, _ = oracle.c1_walk(items, R, seed, mode, grid=GRID)
    s = stream()
    retired = torch.zeros((n, 16), dtype=torch.int32, device=dev())
    with rafi.Context(R, 64, n) as ctx:
        st, cnt, rounds, fwd = rafi.rf_c1_run_graph(ctx.handle, to_dev(items), n, seed, mode, 1.1, GRID, retired,
                                                    deterministic, stream=s)
        assert st == rafi.RF_OK and cnt == n
        assert rounds == int(hops.max()) + 1 and fwd == int(hops.sum())
        got = retired[:cnt].cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(canonical_rows(got), canonical_rows(final))
        k = 4
        want = oracle.c1_rounds(items, R, seed, mode, grid=GRID, dump_round=k)
        st, cnt, rounds, fwd = rafi.rf_c1_run_graph(ctx.handle, to_dev(items), n, seed, mode, 1.1, GRID, retired,
                                                    deterministic, max_rounds=k, stream=s,
                                                    allow=(rafi.RF_ERR_MAX_ROUNDS,))
        assert st == rafi.RF_ERR_MAX_ROUNDS and rounds == k
        assert rafi.rf_num_active(ctx.handle) == int(want["active"][k])
        q, off = _queue(ctx, n, s)
        np.testing.assert_array_equal(off.astype(np.uint64), want["dump_offsets"])
        if deterministic:
            np.testing.assert_array_equal(q, want["dump_items"])
        else:
            for r in range(R):
                np.testing.assert_array_equal(canonical_rows(q[off[r]:off[r + 1]]),
                                              canonical_rows(want["dump_items"][off[r]:off[r + 1]]))


@pytest.mark.parametrize("fuse", [True, False], ids=["step_on_arrival", "step_in_place"])
@pytest.mark.parametrize("ranks,grid,n", [(1, (1, 1, 1), 5000), (1024, (8, 8, 16), 300007), (64, (4, 4, 4), 0),
                                          (64, (4, 4, 4), 17)],
                         ids=["one_rank", "max_ranks", "empty", "ragged"])
def test_batched_rank_count_extremes_and_empty(fuse, ranks, grid, n):
    # one rank (every item forwarded to itself), the maximum rank count (1025
    # destination digits: the per-CTA counts no longer fit one staging pass),
    # an empty run and a run smaller than one tile
    seed = 14
    items = inputs.c1_items(max(n, 1), seed=seed)[:n]
    s = stream()
    retired = torch.zeros((max(n, 1), 16), dtype=torch.int32, device=dev())
    with rafi.Context(ranks, 64, max(n, 1)) as ctx:
        for mode in MODES:
            st, cnt, rounds, fwd = rafi.rf_c1_run_batched(ctx.handle, to_dev(items) if n else retired, n, seed, mode,
                                                          1.1, grid, retired, stream=s, step_on_arrival=fuse)
            assert st == rafi.RF_OK and cnt == n
            if n == 0:
                assert rounds == 0 and fwd == 0 and rafi.rf_num_active(ctx.handle) == 0
                continue
            final, hops, _, _ = oracle.c1_walk(items, ranks, seed, mode, grid=grid)
            assert rounds == int(hops.max()) + 1 and fwd == int(hops.sum())
            got = retired[:cnt].cpu().numpy().view(np.uint32)
            np.testing.assert_array_equal(canonical_rows(got), canonical_rows(final))


_FULL = {}


def _full_items():
    """The bench's 2^24 seeded items (generated once per test session)."""
    if "items" not in _FULL:
        _FULL["items"] = inputs.c1_items(1 << 24, seed=1)
    return _FULL["items"]


def _by_key(a: np.ndarray) -> np.ndarray:
    """Rows ordered by (w0, w1), which identifies an item (checked by the caller)."""
    key = (a[:, 0].astype(np.uint64) << np.uint64(32)) | a[:, 1].astype(np.uint64)
    return a[np.argsort(key, kind="stable")]


@pytest.mark.parametrize("mode", MODES)
def test_full_size_every_word_matches_oracle(mode):
    # The benched configuration, checked word for word: 2^24 x 64 B items over
    # 64 ranks.  The batched forms retire items in the serial round-by-round
    # order (round by round, queue order within a round), so their retirement
    # buffers must equal the oracle's queue simulation row for row, all 16
    # words; the plain host loop appends in scheduling order and is compared
    # as a multiset.  4096 sampled items are also walked one by one.
    n, seed = 1 << 24, 1
    items = _full_items()
    want = oracle.c1_rounds(items, R, seed, mode, grid=GRID)
    want_rounds, want_fwd = int(want["rounds"]), int(want["active"][1:].sum())
    want_items = want["retired_items"]
    d_items = to_dev(items)
    s = stream()
    with rafi.Context(R, 64, n) as ctx:
        ret = torch.zeros((n, 16), dtype=torch.int32, device=dev())
        for fuse in (True, False):
            ret.fill_(-1)
            st, cnt, rounds, fwd = rafi.rf_c1_run_batched(ctx.handle, d_items, n, seed, mode, 1.1, GRID, ret,
                                                          stream=s, step_on_arrival=fuse)
            assert st == rafi.RF_OK and cnt == n
            assert (rounds, fwd) == (want_rounds, want_fwd)
            got = ret.cpu().numpy().view(np.uint32)
            bad = np.flatnonzero(np.any(got != want_items, axis=1))
            assert bad.size == 0, f"step_on_arrival={fuse}: {bad.size} rows differ, first at {bad[:4]}"
        ret.zero_()
        st, cnt, rounds, fwd = rafi.rf_c1_run(ctx.handle, d_items, n, seed, mode, 1.1, GRID, ret, stream=s)
        assert st == rafi.RF_OK and cnt == n and (rounds, fwd) == (want_rounds, want_fwd)
        plain = ret.cpu().numpy().view(np.uint32)
    wk = _by_key(want_items)
    key = (wk[:, 0].astype(np.uint64) << np.uint64(32)) | wk[:, 1].astype(np.uint64)
    assert np.all(np.diff(key) > 0)  # (w0, w1) identifies an item
    np.testing.assert_array_equal(_by_key(plain), wk)
    # sampled items walked one by one through the unpartitioned definition
    sample = np.random.default_rng(mode).choice(n, size=4096, replace=False)
    final, _, unfinished, _ = oracle.c1_walk(items[sample], R, seed, mode, grid=GRID,
                                             start_ranks=(sample % R).astype(np.int32))
    assert unfinished == 0
    skey = (final[:, 0].astype(np.uint64) << np.uint64(32)) | final[:, 1].astype(np.uint64)
    np.testing.assert_array_equal(wk[np.searchsorted(key, skey)], final)


@pytest.mark.parametrize("fuse", [True, False], ids=["step_on_arrival", "step_in_place"])
@pytest.mark.parametrize("mode", MODES)
def test_batched_2m_items_ordered_retirements(mode, fuse):
    # 2^21 items: rounds above 2^20 items and tens of tiles per CTA; the whole
    # retirement buffer equals the oracle's round-by-round order, every word
    n, seed = 1 << 21, 21
    items = inputs.c1_items(n, seed=seed)
    want = oracle.c1_rounds(items, R, seed, mode, grid=GRID)
    got, rounds, fwd, st = _run_batched(items, seed, mode, fuse=fuse)
    assert st == rafi.RF_OK and len(got) == n
    assert rounds == int(want["rounds"]) and fwd == int(want["active"][1:].sum())
    np.testing.assert_array_equal(got, want["retired_items"])


@pytest.mark.parametrize("fuse", [True, False], ids=["step_on_arrival", "step_in_place"])
def test_batched_barrier_timeout_is_reported_and_the_context_recovers(fuse):
    # Each grid barrier waits for one CTA that does not exist, with a bound of
    # 2 * 10^4 cycles: every wait runs out, the abort flag stops every CTA and
    # the call returns RF_ERR_TIMEOUT (no fault, nothing left running).  The
    # same context then runs normally and matches the oracle.
    n, seed = 300007, 31
    items = inputs.c1_items(n, seed=seed)
    final, hops, _, _ = oracle.c1_walk(items, R, seed, rafi.RF_C1_NBR6, grid=GRID)
    with rafi.Context(R, 64, n) as ctx:
        rafi.rf_set_wait_limits(ctx.handle, 20000, 1)
        for _ in range(2):
            got, rounds, fwd, st = _run_batched(items, seed, rafi.RF_C1_NBR6, ctx=ctx, fuse=fuse,
                                                allow=(rafi.RF_ERR_TIMEOUT,))
            assert st == rafi.RF_ERR_TIMEOUT
            assert "gave up" in rafi.rf_last_error()
        rafi.rf_set_wait_limits(ctx.handle, 0, 0)
        got, rounds, fwd, st = _run_batched(items, seed, rafi.RF_C1_NBR6, ctx=ctx, fuse=fuse)
        assert st == rafi.RF_OK and len(got) == n
        assert rounds == int(hops.max()) + 1 and fwd == int(hops.sum())
        np.testing.assert_array_equal(canonical_rows(got), canonical_rows(final))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [20011, 300007, 1 << 20])
def test_batched_retirements_in_the_oracle_order(mode, n):
    # the persistent kernel retires items in the serial round-by-round order:
    # its retirement buffer equals the oracle's queue simulation, every word
    seed = 41
    items = inputs.c1_items(n, seed=seed)
    want = oracle.c1_rounds(items, R, seed, mode, grid=GRID)
    got, rounds, fwd, st = _run_batched(items, seed, mode)
    assert st == rafi.RF_OK and len(got) == n
    assert rounds == int(want["rounds"]) and fwd == int(want["active"][1:].sum())
    np.testing.assert_array_equal(got, want["retired_items"])


@pytest.mark.parametrize("fuse", [True, False], ids=["step_on_arrival", "step_in_place"])
@pytest.mark.parametrize("shape", range(len(rafi.rf_rounds_shapes(rafi.RF_POLICY_MICROBENCH))))
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [20011, 1 << 20])
def test_every_persistent_shape_retires_in_the_oracle_order(mode, shape, n, fuse):
    # each shape the autotuner may pick (threads, tile, CTAs per SM) retires the
    # oracle's items in the oracle's round-by-round order, every word
    seed = 43
    items = inputs.c1_items(n, seed=seed)
    want = oracle.c1_rounds(items, R, seed, mode, grid=GRID)
    with rafi.Context(R, 64, n) as ctx:
        rafi.rf_set_batched_config(ctx.handle, rafi.RF_POLICY_MICROBENCH, rafi.RF_FORM_PERSISTENT, shape)
        assert rafi.rf_get_batched_config(ctx.handle, rafi.RF_POLICY_MICROBENCH) == (rafi.RF_FORM_PERSISTENT, shape)
        got, rounds, fwd, st = _run_batched(items, seed, mode, ctx=ctx, fuse=fuse)
    assert st == rafi.RF_OK and len(got) == n
    assert rounds == int(want["rounds"]) and fwd == int(want["active"][1:].sum())
    np.testing.assert_array_equal(got, want["retired_items"])


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("push", [0, 1024, 1 << 17, 1 << 21, (1 << 32) - 1])
def test_pushed_counts_keep_the_oracle_order(mode, push):
    # Whether a round's counts come from its own count pass or were pushed by
    # the previous scatter (every round of at most `push` items; 2^21 and
    # above push every round after the first, 2^32 - 1 is capped by the
    # kernel), the retirement buffer is the oracle's, every word
    n, seed = 1 << 21, 47
    items = inputs.c1_items(n, seed=seed)
    want = oracle.c1_rounds(items, R, seed, mode, grid=GRID)
    with rafi.Context(R, 64, n) as ctx:
        rafi.rf_set_push_limit(ctx.handle, push)
        assert rafi.rf_get_push_limit(ctx.handle) == push
        got, rounds, fwd, st = _run_batched(items, seed, mode, ctx=ctx)
    assert st == rafi.RF_OK and len(got) == n
    assert rounds == int(want["rounds"]) and fwd == int(want["active"][1:].sum())
    np.testing.assert_array_equal(got, want["retired_items"])


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("skew", [0, 5, 32])
def test_rank_skewed_ranges_keep_the_oracle_order(mode, skew):
    # Large rounds (2^19 items and up) split by SM launch order instead of
    # evenly: the same queues, so the retirement buffer is the oracle's
    n, seed = 1 << 21, 53
    items = inputs.c1_items(n, seed=seed)
    want = oracle.c1_rounds(items, R, seed, mode, grid=GRID)
    with rafi.Context(R, 64, n) as ctx:
        rafi.rf_set_rank_skew(ctx.handle, skew)
        assert rafi.rf_get_rank_skew(ctx.handle) == skew
        with pytest.raises(rafi.RafiError):
            rafi.rf_set_rank_skew(ctx.handle, 33)
        got, rounds, fwd, st = _run_batched(items, seed, mode, ctx=ctx)
    assert st == rafi.RF_OK and len(got) == n
    assert rounds == int(want["rounds"]) and fwd == int(want["active"][1:].sum())
    np.testing.assert_array_equal(got, want["retired_items"])


def test_rank_skew_setup_barrier_timeout_is_reported():
    # the launch-time exchange of SM ids waits at a grid barrier too: with a
    # missing arrival it gives up, and the context then runs normally
    n, seed = 300007, 59
    items = inputs.c1_items(n, seed=seed)
    final, hops, _, _ = oracle.c1_walk(items, R, seed, rafi.RF_C1_UNIFORM, grid=GRID)
    with rafi.Context(R, 64, n) as ctx:
        rafi.rf_set_rank_skew(ctx.handle, 8)
        rafi.rf_set_wait_limits(ctx.handle, 20000, 1)
        got, rounds, fwd, st = _run_batched(items, seed, rafi.RF_C1_UNIFORM, ctx=ctx, allow=(rafi.RF_ERR_TIMEOUT,))
        assert st == rafi.RF_ERR_TIMEOUT
        rafi.rf_set_wait_limits(ctx.handle, 0, 0)
        got, rounds, fwd, st = _run_batched(items, seed, rafi.RF_C1_UNIFORM, ctx=ctx)
        assert st == rafi.RF_OK and len(got) == n
        np.testing.assert_array_equal(canonical_rows(got), canonical_rows(final))
