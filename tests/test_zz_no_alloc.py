"""rf_partition_static: the stable partition for callers that cannot allocate.

Some callers of this library may not call cudaMalloc while they run:
latency-critical loops with a memory budget fixed at start-up (an allocation
can synchronise the device), and hosts whose own caching allocator already
holds nearly all device memory.  For them the library offers one entry point
whose scratch is a fixed static device array.  This file checks it against
the context-based exchange (rf_push + rf_exchange) and against the oracle's
stable partition, bit for bit, on two calls in a row; it is named to run last.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_30294_gb300 import rafi

from gpu_util import dev, exchange_once, stream, to_dev

pytestmark = pytest.mark.gpu


def _static(R, ib, items, dest):
    n = len(dest)
    s = stream()
    out = torch.zeros((max(n, 1), ib), dtype=torch.uint8, device=dev())
    off = torch.zeros(R + 1, dtype=torch.int32, device=dev())
    stats = torch.zeros(4, dtype=torch.int64, device=dev())
    di, dd = to_dev(items), to_dev(dest)
    torch.cuda.synchronize()
    # device-wide free memory can move under another process on a shared GPU,
    # so growth counts as zero when any of a few readings shows none; torch's
    # own pool must not change at all
    grew = []
    reserved = torch.cuda.memory_reserved()
    for _ in range(3):
        free_before = torch.cuda.mem_get_info()[0]
        rafi.rf_partition_static(di, dd, n, ib, R, out, off, stats, s)
        torch.cuda.synchronize()
        grew.append(free_before - torch.cuda.mem_get_info()[0])
    assert torch.cuda.memory_reserved() == reserved
    st = stats.cpu().numpy()
    return out.cpu().numpy(), off.cpu().numpy().astype(np.uint64), st, min(grew)


def test_static_partition_matches_exchange_on_two_calls_in_a_row():
    rng = np.random.default_rng(12)
    # call 1: 64-byte items over 64 ranks, several tiles and a ragged tail
    n1, R1 = 100003, 64
    items1 = rng.integers(0, 256, size=(n1, 64), dtype=np.uint8)
    dest1 = rng.integers(0, R1, size=n1).astype(np.int32)
    # call 2: different shape, with empty slots and invalid destinations
    n2, R2 = 5001, 7
    items2 = rng.integers(0, 256, size=(n2, 48), dtype=np.uint8)
    dest2 = rng.integers(0, R2, size=n2).astype(np.int32)
    dest2[rng.random(n2) < 0.1] = -1
    dest2[rng.random(n2) < 0.02] = 99

    got1, off1, st1, _ = _static(R1, 64, items1, dest1)
    got2, off2, st2, _ = _static(R2, 48, items2, dest2)

    for got, off, st, (R, ib, items, dest) in ((got1, off1, st1, (R1, 64, items1, dest1)),
                                              (got2, off2, st2, (R2, 48, items2, dest2))):
        _, na, want, woff, stats = exchange_once(R, ib, items, dest)
        np.testing.assert_array_equal(off, woff)
        np.testing.assert_array_equal(got[:na], want)
        assert int(st[0]) == na == stats.numActive
        assert int(st[1]) == stats.holes and int(st[2]) == stats.badDest and int(st[3]) == 0
        # and against the oracle's stable partition (Sec. 4.2.1), which shares no code with either
        oout, ooff, obad, oholes = oracle.partition(items, dest, R)
        np.testing.assert_array_equal(off, ooff)
        np.testing.assert_array_equal(got[:len(oout)], oout)
        assert int(st[0]) == len(oout) and int(st[1]) == oholes and int(st[2]) == obad
    # once set up (and its kernels loaded), a call takes no device memory
    got3, off3, st3, grew = _static(R2, 48, items2, dest2)
    assert grew == 0
    np.testing.assert_array_equal(got3, got2)
    np.testing.assert_array_equal(off3, off2)


def test_static_partition_rejects_requests_beyond_its_scratch():
    n, R = 1 << 30, 1024
    with pytest.raises(rafi.RafiError) as e:
        # aligned, non-overlapping stand-in addresses: only the size is wrong, and the
        # library refuses it before touching any of them
        rafi.rf_partition_static(1 << 40, 1 << 39, n, 16, R, 1 << 41, 1 << 38, None, 0)
    assert e.value.status == rafi.RF_ERR_ARG
    assert "static scratch" in rafi.rf_last_error()
