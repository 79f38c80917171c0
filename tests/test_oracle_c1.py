"""Pins for the oracle's forwarding microbenchmark (hop simulator).

The workload is synthetic (64-byte items, retire with probability 0.1 per
hop, destination uniform / Zipf(1.1) / 6-neighbour torus).  What fixes it:
  * the destination laws: closed forms (Hurwitz zeta for Zipf, exact bucket
    boundaries for the uniform and neighbour draws),
  * the retire law: hop counts are geometric(0.1),
  * the payload rule: words 0..12 never change, word 15 counts hops, word 14
    holds the last destination,
  * the forwarding layer: running the workload round by round through the
    oracle's partitioned queues gives exactly the per-item walk's results, and
    items are conserved per round (Sec. 4.2.3's total is the active count).
"""
import numpy as np
import pytest
from scipy import special, stats

import oracle
from paper_2605_30294_gb300 import inputs

R = 64
GRID = (4, 4, 4)


def test_zipf_thresholds_closed_form():
    thr = oracle.zipf_thresholds(R, 1.1)
    assert thr.shape == (R - 1,)
    assert np.all(np.diff(thr.astype(np.int64)) > 0)
    # H = sum_{j=1}^{64} j^-1.1 via Hurwitz zeta: zeta(1.1, 1) - zeta(1.1, 65)
    H = special.zeta(1.1, 1) - special.zeta(1.1, 65)
    p0 = thr[0] / 2**32
    assert abs(p0 - 1.0 / H) < 1e-9
    assert abs(p0 - 0.2505) < 5e-4
    p_last = 1.0 - thr[-1] / 2**32
    assert abs(p_last - 64**-1.1 / H) < 1e-9
    assert abs(p_last - 0.00258) < 5e-5
    for k in (1, 7, 31):
        pk = (int(thr[k]) - int(thr[k - 1])) / 2**32
        assert abs(pk - (k + 1) ** -1.1 / H) < 1e-9


def test_zipf_dest_boundaries():
    thr = oracle.zipf_thresholds(R, 1.1)
    for k in (0, 5, 62):
        assert oracle.choose_dest(oracle.ZIPF, 0, int(thr[k]) - 1, R, thr=thr) == k
        assert oracle.choose_dest(oracle.ZIPF, 0, int(thr[k]), R, thr=thr) == k + 1
    assert oracle.choose_dest(oracle.ZIPF, 0, 2**32 - 1, R, thr=thr) == R - 1
    assert oracle.choose_dest(oracle.ZIPF, 0, 0, R, thr=thr) == 0


@pytest.mark.parametrize("Rr", [1, 3, 64, 512])
def test_uniform_dest_buckets(Rr):
    # d = floor(r1 * R / 2^32): bucket k starts at ceil(k * 2^32 / R)
    for k in range(0, Rr, max(1, Rr // 7)):
        start = -(-k * 2**32 // Rr)
        assert oracle.choose_dest(oracle.UNIFORM, 0, start, Rr) == k
        if start > 0:
            assert oracle.choose_dest(oracle.UNIFORM, 0, start - 1, Rr) == k - 1
    assert oracle.choose_dest(oracle.UNIFORM, 0, 2**32 - 1, Rr) == Rr - 1


def _coords(r):
    return r % 4, (r // 4) % 4, r // 16


def test_nbr6_dest_is_a_torus_neighbour():
    seen = {}
    for src in range(R):
        for k in range(6):
            r1 = -(-k * 2**32 // 6)  # first r1 of direction bucket k
            d = oracle.choose_dest(oracle.NBR6, src, r1, R, grid=GRID)
            a, b = _coords(src), _coords(d)
            diff = [min((x - y) % 4, (y - x) % 4) for x, y in zip(a, b)]
            assert sorted(diff) == [0, 0, 1], (src, k, d)
            seen.setdefault(src, set()).add(d)
    assert all(len(v) == 6 for v in seen.values())
    # +x from (3, y, z) wraps to (0, y, z)
    assert oracle.choose_dest(oracle.NBR6, 3, 0, R, grid=GRID) == 0
    # -z (last bucket) from z = 0 wraps to z = 3
    assert oracle.choose_dest(oracle.NBR6, 5, 2**32 - 1, R, grid=GRID) == 5 + 48


@pytest.mark.parametrize("mode", [oracle.UNIFORM, oracle.ZIPF, oracle.NBR6])
def test_walk_invariants_and_laws(mode):
    n = 1 << 15
    items = inputs.c1_items(n, seed=1)
    final, hops, unfinished, visits = oracle.c1_walk(items, R, 1, mode, grid=GRID, max_hops=400,
                                                     record_visits=True)
    assert unfinished == 0
    # words 0..12 untouched, word 15 counts hops, word 14 is the last destination
    np.testing.assert_array_equal(final[:, :13], items[:, :13])
    np.testing.assert_array_equal(final[:, 15] - items[:, 15], hops)
    moved = hops > 0
    last = visits[np.arange(n), np.maximum(hops.astype(np.int64) - 1, 0)]
    np.testing.assert_array_equal(final[moved, 14], last[moved].astype(np.uint32))
    np.testing.assert_array_equal(final[~moved, 14], items[~moved, 14])
    np.testing.assert_array_equal(final[~moved, 13], items[~moved, 13])
    # hops ~ geometric: P(h = k) = 0.9^k * 0.1, mean 9
    mean = hops.mean()
    assert abs(mean - 9.0) < 5 * np.sqrt(90.0 / n)
    p0 = (hops == 0).mean()
    assert abs(p0 - 0.1) < 5 * np.sqrt(0.09 / n)
    # destination law over all forward events
    v = visits[visits >= 0]
    cnt = np.bincount(v, minlength=R)
    if mode == oracle.UNIFORM:
        exp = np.full(R, v.size / R)
    elif mode == oracle.ZIPF:
        w = np.arange(1, R + 1, dtype=np.float64) ** -1.1
        exp = v.size * w / w.sum()
    else:
        exp = None
    if exp is not None:
        chi2 = ((cnt - exp) ** 2 / exp).sum()
        assert stats.chi2.sf(chi2, R - 1) > 1e-6
    else:
        # every hop moves to a neighbour of the previous rank
        prev = np.concatenate([(np.arange(n) % R)[:, None], visits[:, :-1]], axis=1)
        m = visits >= 0
        a = np.stack(_coords(prev[m]), 1)
        b = np.stack(_coords(visits[m]), 1)
        diff = np.minimum((a - b) % 4, (b - a) % 4)
        assert np.all(np.sort(diff, 1) == np.array([0, 0, 1]))


def test_payload_update_word_is_independent_of_retire_and_destination_words():
    # For one-hop items w13 ^ w13_0 is the update word of that hop.  It must be
    # uniform on [0, 2^32) (not the retire word, which is >= the threshold for a
    # forwarded item) and independent of the destination (not the destination word).
    n = 1 << 16
    items = inputs.c1_items(n, seed=2)
    final, hops, _, _ = oracle.c1_walk(items, R, 2, oracle.UNIFORM)
    one = hops == 1
    x = final[one, 13] ^ items[one, 13]
    below = (x < oracle.RETIRE_THRESHOLD).mean()
    assert abs(below - 0.1) < 5 * np.sqrt(0.09 / one.sum())
    top = (x >> 26).astype(np.int64)
    agree = (top == final[one, 14].astype(np.int64)).mean()
    assert agree < 1.0 / R + 5 * np.sqrt(1.0 / (R * one.sum()))


def test_retire_threshold_is_a_tenth():
    assert oracle.RETIRE_THRESHOLD == int(np.ceil(0.1 * 2**32))


@pytest.mark.parametrize("mode", [oracle.UNIFORM, oracle.ZIPF, oracle.NBR6])
def test_rounds_equal_walk(mode):
    n = 5000
    items = inputs.c1_items(n, seed=11)
    final, hops, _, _ = oracle.c1_walk(items, R, 11, mode, grid=GRID)
    res = oracle.c1_rounds(items, R, 11, mode, grid=GRID)
    # rounds run = 1 + the largest hop count; the retired multiset is the walk's
    assert res["rounds"] == int(hops.max()) + 1
    a = res["retired_items"]
    key = lambda x: np.lexsort(x.T[::-1])
    np.testing.assert_array_equal(a[key(a)], final[key(final)])
    # conservation per round: active_k = retired_k + active_{k+1}
    act, ret = res["active"], res["retired"]
    assert int(act[0]) == n and int(act[-1]) == 0
    np.testing.assert_array_equal(act[:-1], ret + act[1:])
    # the number retiring in round k is the number of items with k hops
    np.testing.assert_array_equal(ret, np.bincount(hops, minlength=res["rounds"]))


def test_round_zero_queue_is_stable():
    n = 1000
    items = inputs.c1_items(n, seed=5)
    res = oracle.c1_rounds(items, R, 5, oracle.UNIFORM, dump_round=0)
    off = res["dump_offsets"].astype(np.int64)
    q = res["dump_items"]
    for r in (0, 1, 39, 63):
        idx = np.arange(r, n, R)
        np.testing.assert_array_equal(q[off[r]:off[r + 1]], items[idx])


def test_round_queues_hold_the_walk_positions():
    # at round k, rank r's queue holds exactly the items whose k-th position is r
    n, k = 3000, 3
    items = inputs.c1_items(n, seed=9)
    _, hops, _, visits = oracle.c1_walk(items, R, 9, oracle.ZIPF, max_hops=400, record_visits=True)
    res = oracle.c1_rounds(items, R, 9, oracle.ZIPF, dump_round=k)
    off = res["dump_offsets"].astype(np.int64)
    alive = np.nonzero(hops >= k)[0]
    pos = visits[alive, k - 1]
    for r in range(R):
        q = res["dump_items"][off[r]:off[r + 1]]
        want = items[alive[pos == r], :2]
        got = q[:, :2]
        assert sorted(map(tuple, got)) == sorted(map(tuple, want))
