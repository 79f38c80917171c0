"""Pins for the oracle's exchange (stable partition by destination).

The paper's exchange radix-sorts keys (dest << 32 | i) and gathers the items
in key order (Sec. 4.2.1), then hands each rank its contiguous block
(Sec. 4.2.2).  Brute force: Python's stable ``sorted`` on the destination and
numpy's stable argsort give the same permutation.
"""
import numpy as np
import pytest

import oracle


def _brute(items, dest, R):
    keep = [i for i in range(len(dest)) if 0 <= dest[i] < R]
    order = sorted(keep, key=lambda i: int(dest[i]))
    out = items[order] if order else items[:0]
    off = np.zeros(R + 1, np.uint64)
    for d in dest:
        if 0 <= d < R:
            off[d + 1] += 1
    return out, np.cumsum(off).astype(np.uint64)


def _key_sort(items, dest, R):
    # the paper's formulation: sort 64-bit keys dest<<32 | i, gather by key
    valid = np.nonzero((dest >= 0) & (dest < R))[0]
    keys = (dest[valid].astype(np.uint64) << np.uint64(32)) | valid.astype(np.uint64)
    keys.sort()
    idx = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    return items[idx]


CASES = [
    ("random", 1000, 3, 16),
    ("random", 777, 64, 64),
    ("random", 513, 512, 48),
    ("random", 300, 2, 128),
    ("one_rank", 200, 1, 16),
]


@pytest.mark.parametrize("kind,n,R,ib", CASES)
def test_partition_matches_brute_force(kind, n, R, ib):
    rng = np.random.default_rng(n * 31 + R)
    items = rng.integers(0, 256, size=(n, ib), dtype=np.uint8)
    dest = rng.integers(0, R, size=n).astype(np.int32)
    out, off, bad, holes = oracle.partition(items, dest, R)
    bo, boff = _brute(items, dest, R)
    np.testing.assert_array_equal(out, bo)
    np.testing.assert_array_equal(off, boff)
    np.testing.assert_array_equal(out, _key_sort(items, dest, R))
    assert bad == 0 and holes == 0


def test_partition_all_to_one_rank_keeps_order():
    n, R = 100, 64
    items = np.arange(n * 16, dtype=np.uint32).view(np.uint8).reshape(n, 64)
    dest = np.full(n, 17, np.int32)
    out, off, _, _ = oracle.partition(items, dest, R)
    np.testing.assert_array_equal(out, items)
    assert int(off[17]) == 0 and int(off[18]) == n and int(off[-1]) == n
    assert all(int(off[r]) == 0 for r in range(18)) and all(int(off[r]) == n for r in range(18, R + 1))


def test_partition_empty_and_empty_ranks():
    out, off, bad, holes = oracle.partition(np.zeros((0, 16), np.uint8), np.zeros(0, np.int32), 5)
    assert out.shape == (0, 16) and np.all(off == 0) and bad == 0 and holes == 0
    # ranks 0, 2, 4 receive nothing
    items = np.arange(6 * 16, dtype=np.uint8).reshape(6, 16)
    dest = np.array([3, 1, 3, 1, 1, 3], np.int32)
    out, off, _, _ = oracle.partition(items, dest, 5)
    assert list(off) == [0, 0, 3, 3, 6, 6]
    np.testing.assert_array_equal(out, items[[1, 3, 4, 0, 2, 5]])


def test_partition_holes_and_bad_destinations():
    items = np.arange(8 * 16, dtype=np.uint8).reshape(8, 16)
    dest = np.array([0, -1, 2, 7, -5, 1, -1, 0], np.int32)
    out, off, bad, holes = oracle.partition(items, dest, 3)
    assert holes == 2 and bad == 2
    assert list(off) == [0, 2, 3, 4]
    np.testing.assert_array_equal(out, items[[0, 7, 5, 2]])


def test_partition_identity_when_sorted():
    # input already grouped by destination: the partition is the identity
    n, R = 4096, 64
    dest = np.sort(np.random.default_rng(1).integers(0, R, n)).astype(np.int32)
    items = np.random.default_rng(2).integers(0, 256, (n, 32), dtype=np.uint8)
    out, off, _, _ = oracle.partition(items, dest, R)
    np.testing.assert_array_equal(out, items)
    np.testing.assert_array_equal(off[:-1], np.searchsorted(dest, np.arange(R)).astype(np.uint64))


def test_joint_runs_partition_restricted_to_a_run_is_that_runs_own():
    # Several independent runs can share one round's queue (the batched form's
    # joint launch): each item moves by a rule of its own bytes and the round,
    # never of its position.  Then the stable partition of the joint queue,
    # restricted to one run's items, is that run's own stable partition, round
    # after round, and so are the items each round retires, in order.
    rng = np.random.default_rng(7)
    R, K, n, ib = 16, 3, 500, 16
    runs = []
    for k in range(K):
        it = rng.integers(0, 256, size=(n, ib), dtype=np.uint8)
        it[:, 0] = k  # run tag (the rule below ignores it)
        it[:, 1:5] = np.arange(n, dtype=np.uint32).view(np.uint8).reshape(n, 4)  # unique per run
        runs.append(it)

    def rule(items, rnd):
        # next destination from the item's bytes 5.. and the round; -1 retires
        h = (items[:, 5:].astype(np.uint64) * np.arange(1, ib - 4, dtype=np.uint64)).sum(axis=1)
        h = (h * np.uint64(2654435761) + np.uint64(rnd * 40503)) % np.uint64(1 << 31)
        d = (h % np.uint64(R + 3)).astype(np.int32)
        return np.where(d >= R, -1, d)

    def first(items):  # item i of a run starts at rank i mod R
        return (items[:, 1:5].copy().view(np.uint32)[:, 0] % R).astype(np.int32)

    joint, _, _, _ = oracle.partition(np.concatenate(runs), np.concatenate([first(r) for r in runs]), R)
    own = [oracle.partition(r, first(r), R)[0] for r in runs]
    for rnd in range(12):
        for k in range(K):
            np.testing.assert_array_equal(joint[joint[:, 0] == k], own[k])
        dj = rule(joint, rnd)
        retired_joint = joint[dj < 0]
        joint = oracle.partition(joint, dj, R)[0]
        for k in range(K):
            dk = rule(own[k], rnd)
            np.testing.assert_array_equal(retired_joint[retired_joint[:, 0] == k], own[k][dk < 0])
            own[k] = oracle.partition(own[k], dk, R)[0]
    assert len(joint) < K * n  # items did retire along the way
