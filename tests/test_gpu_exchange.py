"""GPU parity: rf_exchange (count / scan / stable scatter) against the oracle.

Items pushed from the host side keep their push order in the out-queue, so
the exchange result is compared bit-exactly with the oracle's stable
partition (Sec. 4.2.1-4.2.3): same items, same order, same segment offsets.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_30294_gb300 import rafi

from gpu_util import exchange_once, stream, to_dev, zeros_u8

pytestmark = pytest.mark.gpu

CASES = [
    # (numRanks, itemBytes, n) -- spans several tiles with a ragged tail
    (1, 64, 5000),
    (2, 16, 10007),
    (3, 48, 3001),
    (64, 64, (1 << 16) + 123),
    (64, 128, 7777),
    (64, 96, 4099),      # generic vector count (6 vectors per item)
    (512, 64, 100003),
    (1024, 16, 50001),
    (8, 512, 1000),
    (64, 64, 1),
    (7, 32, 255),
]


def _items(n, ib, seed):
    return np.random.default_rng(seed).integers(0, 256, size=(n, ib), dtype=np.uint8)


@pytest.mark.parametrize("R,ib,n", CASES)
def test_exchange_uniform_matches_oracle(R, ib, n):
    rng = np.random.default_rng(R * 7 + n)
    items = _items(n, ib, n)
    dest = rng.integers(0, R, size=n).astype(np.int32)
    st, na, got, off, stats = exchange_once(R, ib, items, dest)
    want, woff, bad, holes = oracle.partition(items, dest, R)
    assert st == rafi.RF_OK and na == n
    np.testing.assert_array_equal(off, woff)
    np.testing.assert_array_equal(got, want)
    assert stats.numActive == n and stats.emitted == n and stats.dropped == 0 and stats.badDest == 0


@pytest.mark.parametrize("R", [64, 1024])
def test_exchange_zipf_skew(R):
    n = 200000
    rng = np.random.default_rng(3)
    w = np.arange(1, R + 1, dtype=np.float64) ** -1.1
    dest = rng.choice(R, size=n, p=w / w.sum()).astype(np.int32)
    items = _items(n, 64, 5)
    st, na, got, off, _ = exchange_once(R, 64, items, dest)
    want, woff, _, _ = oracle.partition(items, dest, R)
    np.testing.assert_array_equal(off, woff)
    np.testing.assert_array_equal(got, want)


def test_exchange_all_to_one_rank_and_empty_ranks():
    n, R = 40000, 64
    items = _items(n, 64, 11)
    dest = np.full(n, 37, np.int32)
    st, na, got, off, _ = exchange_once(R, 64, items, dest)
    np.testing.assert_array_equal(got, items)
    assert list(off[:38]) == [0] * 38 and list(off[38:]) == [n] * (R + 1 - 38)


def test_exchange_empty():
    st, na, got, off, stats = exchange_once(16, 64, np.zeros((0, 64), np.uint8), np.zeros(0, np.int32))
    assert st == rafi.RF_OK and na == 0 and np.all(off == 0)
    assert stats.exchanges == 1 and stats.totalDelivered == 0


def test_exchange_holes_and_bad_destinations():
    n, R = 30000, 32
    rng = np.random.default_rng(8)
    dest = rng.integers(0, R, size=n).astype(np.int32)
    dest[rng.random(n) < 0.2] = -1
    badmask = rng.random(n) < 0.01
    dest[badmask] = rng.choice([-7, R, R + 5, 2**31 - 1], size=badmask.sum())
    items = _items(n, 48, 9)
    st, na, got, off, stats = exchange_once(R, 48, items, dest)
    want, woff, bad, holes = oracle.partition(items, dest, R)
    assert st == rafi.RF_ERR_BAD_DEST
    assert stats.badDest == bad and stats.holes == holes and na == len(want)
    np.testing.assert_array_equal(off, woff)
    np.testing.assert_array_equal(got, want)


def test_exchange_overflow_drops_and_reports():
    R, cap, n = 16, 5000, 7000
    items = _items(n, 64, 1)
    dest = np.random.default_rng(2).integers(0, R, size=n).astype(np.int32)
    s = stream()
    with rafi.Context(R, 64, cap) as ctx:
        # two pushes: the second one only partly fits
        rafi.rf_push(ctx.handle, to_dev(items[:4000]), to_dev(dest[:4000]), 4000, False, s)
        rafi.rf_push(ctx.handle, to_dev(items[4000:]), to_dev(dest[4000:]), n - 4000, False, s)
        st, na = rafi.rf_exchange(ctx.handle, s, allow=(rafi.RF_ERR_OVERFLOW,))
        assert st == rafi.RF_ERR_OVERFLOW and na == cap
        stats = rafi.rf_stats(ctx.handle, allow=(rafi.RF_ERR_OVERFLOW,))
        assert stats.dropped == n - cap and stats.emitted == cap
        out = zeros_u8(cap, 64)
        off = torch.zeros(R + 1, dtype=torch.int32, device=out.device)
        rafi.rf_snapshot(ctx.handle, out, off, s, allow=(rafi.RF_ERR_OVERFLOW,))
        want, woff, _, _ = oracle.partition(items[:cap], dest[:cap], R)
        np.testing.assert_array_equal(out.cpu().numpy(), want)
        # the next exchange starts clean
        st, na = rafi.rf_exchange(ctx.handle, s)
        assert st == rafi.RF_OK and na == 0


def test_exchange_host_push_and_repeated_rounds():
    R, ib = 10, 32
    s = stream()
    with rafi.Context(R, ib, 20000) as ctx:
        total = 0
        for k, n in enumerate([12345, 1, 0, 19999]):
            items = _items(n, ib, 100 + k)
            dest = np.random.default_rng(k).integers(0, R, size=n).astype(np.int32)
            if n:
                rafi.rf_push(ctx.handle, items.ctypes.data, dest.ctypes.data, n, True, s)
            st, na = rafi.rf_exchange(ctx.handle, s)
            assert st == rafi.RF_OK and na == n
            total += n
            out = zeros_u8(20000, ib)
            off = torch.zeros(R + 1, dtype=torch.int32, device=out.device)
            rafi.rf_snapshot(ctx.handle, out, off, s)
            want, woff, _, _ = oracle.partition(items, dest, R)
            np.testing.assert_array_equal(out[:n].cpu().numpy(), want)
            for r in (0, R // 2, R - 1):
                o, c = rafi.rf_segment(ctx.handle, r)
                assert (o, c) == (int(woff[r]), int(woff[r + 1] - woff[r]))
        stats = rafi.rf_stats(ctx.handle)
        assert stats.exchanges == 4 and stats.totalDelivered == total


def test_snapshot_restore_roundtrip():
    R, ib, n = 12, 64, 9000
    items = _items(n, ib, 4)
    dest = np.random.default_rng(4).integers(0, R, size=n).astype(np.int32)
    s = stream()
    with rafi.Context(R, ib, n) as a, rafi.Context(R, ib, n) as b:
        rafi.rf_push(a.handle, to_dev(items), to_dev(dest), n, False, s)
        rafi.rf_exchange(a.handle, s)
        q = zeros_u8(n, ib)
        off = torch.zeros(R + 1, dtype=torch.int32, device=q.device)
        rafi.rf_snapshot(a.handle, q, off, s)
        rafi.rf_restore(b.handle, q, off, n, s)
        assert rafi.rf_num_active(b.handle) == n
        q2 = zeros_u8(n, ib)
        off2 = torch.zeros(R + 1, dtype=torch.int32, device=q.device)
        rafi.rf_snapshot(b.handle, q2, off2, s)
        torch.cuda.synchronize()
        assert torch.equal(q, q2) and torch.equal(off, off2)
        assert rafi.rf_segment(b.handle, 5) == rafi.rf_segment(a.handle, 5)


def test_device_queue_interface_fields():
    with rafi.Context(5, 48, 1234) as ctx:
        q = rafi.rf_get_device_queues(ctx.handle)
        assert q.capacity == 1234 and q.itemBytes == 48 and q.numRanks == 5
        assert q.in_ and q.out and q.dest and q.outCount and q.inOffset
        assert q.in_ % 16 == 0 and q.out % 16 == 0


def test_timing_counters():
    R, n = 64, 1 << 20
    items = _items(n, 64, 6)
    dest = np.random.default_rng(6).integers(0, R, size=n).astype(np.int32)
    s = stream()
    with rafi.Context(R, 64, n) as ctx:
        rafi.rf_set_timing(ctx.handle, True)
        launches = rafi.rf_launch_count()
        rafi.rf_push(ctx.handle, to_dev(items), to_dev(dest), n, False, s)
        rafi.rf_exchange(ctx.handle, s)
        t = rafi.rf_get_timing(ctx.handle, reset=True)
        assert t.scatterLaunches == 1 and t.scatterItems == n and t.scatterMs > 0
        assert t.scatterLaunchesLarge == 1 and t.scatterItemsLarge == n
        assert rafi.rf_launch_count() - launches == 5  # add_count + count + scan + scatter + wrap-up


# ---------------------------------------------------------------------------
# exchange configuration and autotuner
# ---------------------------------------------------------------------------
TILES = {16: (4096, 2048, 1024), 32: (2048, 1024, 512), 48: (1024, 512, 256), 64: (1024, 512, 256),
         128: (512, 256)}


def _exchange_with(ctx, R, ib, items, dest, s):
    n = len(dest)
    rafi.rf_push(ctx.handle, to_dev(items), to_dev(dest), n, False, s)
    st, na = rafi.rf_exchange(ctx.handle, s)
    out = zeros_u8(n, ib)
    off = torch.zeros(R + 1, dtype=torch.int32, device=torch.device("cuda:0"))
    rafi.rf_snapshot(ctx.handle, out, off, s)
    torch.cuda.synchronize()
    return na, out[:na].cpu().numpy(), off.cpu().numpy().astype(np.uint64)


@pytest.mark.parametrize("ib", sorted(TILES))
def test_every_exchange_config_gives_the_stable_partition(ib):
    R, n = 64, 100003
    rng = np.random.default_rng(ib)
    items = _items(n, ib, ib + 1)
    dest = rng.integers(0, R, size=n).astype(np.int32)
    want, woff, _, _ = oracle.partition(items, dest, R)
    s = stream()
    with rafi.Context(R, ib, n) as ctx:
        default = rafi.rf_get_exchange_config(ctx.handle)
        assert default[0] == TILES[ib][0]
        for tile in TILES[ib]:
            for grid in (0, 7, 152):
                rafi.rf_set_exchange_config(ctx.handle, tile, grid, grid)
                assert rafi.rf_get_exchange_config(ctx.handle)[0] == tile
                na, got, off = _exchange_with(ctx, R, ib, items, dest, s)
                assert na == n
                np.testing.assert_array_equal(off, woff)
                np.testing.assert_array_equal(got, want)
        # a tile no variant has is refused and leaves the configuration as it was
        before = rafi.rf_get_exchange_config(ctx.handle)
        st = rafi.rf_set_exchange_config(ctx.handle, 256 * 3, 0, 0, allow=(rafi.RF_ERR_ARG,))
        assert st == rafi.RF_ERR_ARG and rafi.rf_get_exchange_config(ctx.handle) == before


def test_tuner_keeps_the_out_queue_and_picks_a_variant():
    R, ib, n = 64, 64, 1 << 20
    rng = np.random.default_rng(11)
    items = _items(n, ib, 12)
    dest = rng.integers(0, R, size=n).astype(np.int32)
    want, woff, _, _ = oracle.partition(items, dest, R)
    s = stream()
    with rafi.Context(R, ib, n) as ctx:
        rafi.rf_push(ctx.handle, to_dev(items), to_dev(dest), n, False, s)
        cfg, ms = rafi.rf_tune_exchange(ctx.handle, s, trials=2)
        assert cfg[0] in TILES[ib] and cfg[1] > 0 and ms > 0
        assert rafi.rf_get_exchange_config(ctx.handle) == cfg
        assert rafi.rf_num_active(ctx.handle) == 0  # the incoming queue is left empty
        st, na = rafi.rf_exchange(ctx.handle, s)
        out = zeros_u8(n, ib)
        off = torch.zeros(R + 1, dtype=torch.int32, device=torch.device("cuda:0"))
        rafi.rf_snapshot(ctx.handle, out, off, s)
        torch.cuda.synchronize()
        assert na == n
        np.testing.assert_array_equal(off.cpu().numpy().astype(np.uint64), woff)
        np.testing.assert_array_equal(out.cpu().numpy(), want)
        # an empty out-queue has nothing to tune on
        with pytest.raises(rafi.RafiError):
            rafi.rf_tune_exchange(ctx.handle, s)


def test_context_over_caller_owned_queues():
    R, ib, n = 64, 64, 30011
    rng = np.random.default_rng(21)
    items = _items(n, ib, 22)
    dest = rng.integers(0, R, size=n).astype(np.int32)
    want, woff, _, _ = oracle.partition(items, dest, R)
    cuda = torch.device("cuda:0")
    q_in = torch.zeros((n, ib), dtype=torch.uint8, device=cuda)
    q_out = torch.zeros((n, ib), dtype=torch.uint8, device=cuda)
    q_dest = torch.zeros((n + 3) // 4 * 4 + 4, dtype=torch.int32, device=cuda)
    s = stream()
    with rafi.Context(R, ib, n, buffers=(q_in, q_out, q_dest)) as ctx:
        q = rafi.rf_get_device_queues(ctx.handle)
        assert (q.in_, q.out, q.dest) == (q_in.data_ptr(), q_out.data_ptr(), q_dest.data_ptr())
        na, got, off = _exchange_with(ctx, R, ib, items, dest, s)
        assert na == n
        np.testing.assert_array_equal(off, woff)
        np.testing.assert_array_equal(got, want)
        # the delivered queue is the caller's tensor
        np.testing.assert_array_equal(q_in.cpu().numpy(), want)
        with pytest.raises(rafi.RafiError):
            rafi.rf_resize(ctx.handle, 2 * n)
    # destroying the context leaves the caller's buffers usable
    q_in.fill_(7)
    torch.cuda.synchronize()
    assert int(q_in[0, 0]) == 7
    with pytest.raises(rafi.RafiError):
        rafi.rf_create_with_buffers(R, ib, n, q_in[:, 1:], q_out, q_dest)  # misaligned
