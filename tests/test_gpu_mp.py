"""GPU parity: the multi-phase exchange with three contexts on one stream.

A particle context (32-byte items), a node context (64-byte items) and a
request context (16-byte items) share one stream, as the paper's N-body code
drives three forwarding contexts (Sec. 5.5).  Every phase is compared with
the oracle exactly (the workload is integer-only): per rank, the multiset of
incoming items after each exchange, and the local-tree nodes word by word.
Queue order within a rank is an atomic-append order, so rows are compared
after a canonical sort.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_30294_gb300 import inputs, rafi

from gpu_util import canonical_rows, dev, stream, to_dev

pytestmark = pytest.mark.gpu

GRID = (4, 4, 4)
R = 64


def _incoming(ctx, item_words, cap, s):
    q = torch.zeros((max(cap, 1), item_words), dtype=torch.int32, device=dev())
    off = torch.zeros(R + 1, dtype=torch.int32, device=dev())
    rafi.rf_snapshot(ctx.handle, q, off, s)
    torch.cuda.synchronize()
    o = off.cpu().numpy().astype(np.int64)
    rows = q.cpu().numpy().view(np.uint32)
    return [rows[o[r]:o[r + 1]] for r in range(R)]


def _same_per_rank(got, want):
    assert len(got) == len(want)
    for r in range(len(want)):
        np.testing.assert_array_equal(canonical_rows(got[r]), canonical_rows(np.asarray(want[r], np.uint32)),
                                      err_msg=f"rank {r}")


def _contexts(n):
    roots = R * (R - 1)
    return (rafi.Context(R, 32, n), rafi.Context(R, 64, roots + R * 26 * 8), rafi.Context(R, 16, R * 26))


def _seed(pc, particles, s):
    rafi.rf_mp_seed(pc.handle, to_dev(particles), len(particles), GRID, stream=s)
    rafi.rf_exchange(pc.handle, s)


@pytest.mark.parametrize("n", [20, 3000, 200003])
def test_each_phase_matches_oracle(n):
    p = inputs.mp_particles(n, seed=7)
    want = oracle.mp_protocol(p, GRID)
    s = stream()
    nodes = torch.zeros((R, 9, 5), dtype=torch.int64, device=dev())
    pc, nc, rc = _contexts(n)
    with pc, nc, rc:
        _seed(pc, p, s)
        _, owner0 = oracle.mp_migrate(np.concatenate([p[:, :3], np.zeros((n, 5), np.uint32)], axis=1), GRID)
        _same_per_rank(_incoming(pc, 8, n, s), [p[owner0 == r] for r in range(R)])

        rafi.rf_mp_migrate(pc.handle, GRID, stream=s)
        rafi.rf_exchange(pc.handle, s)
        _same_per_rank(_incoming(pc, 8, n, s), want["particles_at"])

        rafi.rf_mp_tree(pc.handle, GRID, nodes, stream=s)
        np.testing.assert_array_equal(nodes.cpu().numpy().view(np.uint64), want["nodes"])

        rafi.rf_mp_broadcast(nc.handle, nodes, stream=s)
        _, na = rafi.rf_exchange(nc.handle, s)
        assert na == R * (R - 1)
        _same_per_rank(_incoming(nc, 16, R * (R - 1), s), want["roots_at"])

        rafi.rf_mp_request(nc.handle, rc.handle, GRID, stream=s)
        _, nq = rafi.rf_exchange(rc.handle, s)
        assert nq == sum(len(a) for a in want["requests_at"])
        _same_per_rank(_incoming(rc, 4, max(nq, 1), s), want["requests_at"])

        rafi.rf_mp_respond(rc.handle, nc.handle, nodes, stream=s)
        _, nch = rafi.rf_exchange(nc.handle, s)
        assert nch == sum(len(a) for a in want["children_at"])
        _same_per_rank(_incoming(nc, 16, max(nch, 1), s), want["children_at"])


def test_two_steps_through_one_call():
    n = 50000
    p = inputs.mp_particles(n, seed=8, speed_bits=28)
    first = oracle.mp_protocol(p, GRID)
    second = oracle.mp_protocol(first["moved"], GRID)
    s = stream()
    nodes = torch.zeros((R, 9, 5), dtype=torch.int64, device=dev())
    pc, nc, rc = _contexts(n)
    with pc, nc, rc:
        _seed(pc, p, s)
        got1 = rafi.rf_mp_step(pc.handle, nc.handle, rc.handle, GRID, nodes, stream=s)
        assert got1 == (n, R * (R - 1), sum(len(a) for a in first["requests_at"]),
                        sum(len(a) for a in first["children_at"]))
        got2 = rafi.rf_mp_step(pc.handle, nc.handle, rc.handle, GRID, nodes, stream=s)
        assert got2[0] == n and got2[1] == R * (R - 1)
        np.testing.assert_array_equal(nodes.cpu().numpy().view(np.uint64), second["nodes"])
        _same_per_rank(_incoming(pc, 8, n, s), second["particles_at"])
        _same_per_rank(_incoming(nc, 16, got2[3], s), second["children_at"])


def test_contexts_interleave_on_one_stream():
    # the particle exchange of the next step is issued between the node and
    # request phases of this one: contexts never share queues or counters
    n = 4000
    p = inputs.mp_particles(n, seed=9)
    first = oracle.mp_protocol(p, GRID)
    second = oracle.mp_protocol(first["moved"], GRID)
    s = stream()
    nodes = torch.zeros((R, 9, 5), dtype=torch.int64, device=dev())
    pc, nc, rc = _contexts(n)
    with pc, nc, rc:
        _seed(pc, p, s)
        rafi.rf_mp_migrate(pc.handle, GRID, stream=s)
        rafi.rf_exchange(pc.handle, s)
        rafi.rf_mp_tree(pc.handle, GRID, nodes, stream=s)
        rafi.rf_mp_broadcast(nc.handle, nodes, stream=s)
        rafi.rf_mp_migrate(pc.handle, GRID, stream=s)  # next step's migration, in between
        rafi.rf_exchange(nc.handle, s)
        rafi.rf_exchange(pc.handle, s)
        rafi.rf_mp_request(nc.handle, rc.handle, GRID, stream=s)
        rafi.rf_exchange(rc.handle, s)
        _same_per_rank(_incoming(pc, 8, n, s), second["particles_at"])
        _same_per_rank(_incoming(rc, 4, R * 26, s), first["requests_at"])
