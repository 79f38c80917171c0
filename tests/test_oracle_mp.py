"""Pins for the oracle's multi-phase exchange (Sec. 5.5's protocol: particle
migration, root broadcast, refinement requests, child replies).

  * ownership: the corners of every rank's box belong to it, one box width
    along an axis is the next rank along it (with wrap-around), and every
    point of a brute-force sample lies inside its owner's box;
  * migration is exact modular motion: moving with -v undoes it, mass and id
    are kept;
  * the trees conserve mass, weighted coordinates and count (the roots sum to
    the whole set, each root is the sum of its eight octants), checked with
    Python integers on a brute-force sample;
  * nearness: symmetric, 26 neighbours on 4^3 and 8^3 tori, every other rank
    on 2^3;
  * the protocol's item counts have their closed forms.
"""
import numpy as np

import oracle
from paper_2605_30294_gb300 import inputs

GRID = (4, 4, 4)


def test_owner_boxes():
    for grid in ((4, 4, 4), (2, 4, 8), (8, 8, 8)):
        gx, gy, gz = grid
        wx, wy, wz = 2 ** 32 // gx, 2 ** 32 // gy, 2 ** 32 // gz
        for r in range(gx * gy * gz):
            bx, by, bz = r % gx, (r // gx) % gy, r // (gx * gy)
            for dx in (0, wx - 1):
                for dy in (0, wy - 1):
                    for dz in (0, wz - 1):
                        assert oracle.mp_owner(bx * wx + dx, by * wy + dy, bz * wz + dz, grid) == r
        # one box width along x is the next rank along x, wrapping
        assert oracle.mp_owner((gx - 1) * wx, 0, 0, grid) == gx - 1
        assert oracle.mp_owner(((gx - 1) * wx + wx) % 2 ** 32, 0, 0, grid) == 0
    rng = np.random.default_rng(1)
    for x, y, z in rng.integers(0, 2 ** 32, size=(500, 3)):
        r = oracle.mp_owner(int(x), int(y), int(z), GRID)
        bx, by, bz = r % 4, (r // 4) % 4, r // 16
        assert bx * 2 ** 30 <= x < (bx + 1) * 2 ** 30
        assert by * 2 ** 30 <= y < (by + 1) * 2 ** 30
        assert bz * 2 ** 30 <= z < (bz + 1) * 2 ** 30


def test_migration_is_exact_modular_motion():
    p = inputs.mp_particles(5000)
    moved, owner = oracle.mp_migrate(p, GRID)
    back = moved.copy()
    back[:, 3:6] = (-(p[:, 3:6].view(np.int32).astype(np.int64))).astype(np.int32).view(np.uint32)
    undone, _ = oracle.mp_migrate(back, GRID)
    np.testing.assert_array_equal(undone[:, :3], p[:, :3])
    np.testing.assert_array_equal(moved[:, 3:], p[:, 3:])
    want = (p[:, :3].astype(np.int64) + p[:, 3:6].view(np.int32)) % 2 ** 32
    np.testing.assert_array_equal(moved[:, :3], want.astype(np.uint32))
    for i in range(0, 5000, 97):
        assert owner[i] == oracle.mp_owner(*(int(v) for v in moved[i, :3]), GRID)
    # about the expected share leaves its box: speed 2^26 against box width 2^30
    assert 0.01 < np.mean(owner != [oracle.mp_owner(*(int(v) for v in q[:3]), GRID) for q in p]) < 0.2


def test_trees_conserve_brute_force():
    p = inputs.mp_particles(3000, seed=9)
    nodes = oracle.mp_tree(p, GRID)
    R = 64
    want = [[0] * 5 for _ in range(R)]
    octs = [[[0] * 5 for _ in range(8)] for _ in range(R)]
    for q in p:
        x, y, z, m = int(q[0]), int(q[1]), int(q[2]), int(q[6])
        r = (x >> 30) + 4 * ((y >> 30) + 4 * (z >> 30))
        o = ((x >> 29) & 1) | (((y >> 29) & 1) << 1) | (((z >> 29) & 1) << 2)
        for acc in (want[r], octs[r][o]):
            acc[0] += m
            acc[1] += m * x
            acc[2] += m * y
            acc[3] += m * z
            acc[4] += 1
    for r in range(R):
        assert [int(v) for v in nodes[r, 0]] == want[r]
        for o in range(8):
            assert [int(v) for v in nodes[r, 1 + o]] == octs[r][o]
    assert int(nodes[:, 0, 0].sum()) == int(p[:, 6].astype(np.int64).sum())
    assert int(nodes[:, 0, 4].sum()) == len(p)
    np.testing.assert_array_equal(nodes[:, 0], nodes[:, 1:].sum(axis=1))


def test_nearness():
    for grid, k in (((4, 4, 4), 26), ((8, 8, 8), 26), ((2, 2, 2), 7)):
        R = int(np.prod(grid))
        near = np.array([[oracle.mp_near(r, s, grid) for s in range(R)] for r in range(R)])
        assert (near == near.T).all() and not near.diagonal().any()
        assert (near.sum(axis=1) == k).all()


def test_protocol_counts():
    p = inputs.mp_particles(20000)
    out = oracle.mp_protocol(p, GRID)
    R = 64
    nodes = out["nodes"]
    assert all(len(a) == R - 1 for a in out["roots_at"])
    assert sum(len(a) for a in out["particles_at"]) == len(p)
    nonempty = nodes[:, 0, 4] > 0
    assert nonempty.all()  # 20000 particles over 64 ranks
    assert all(len(a) == 26 for a in out["requests_at"])
    # each rank receives the non-empty octants of its 26 neighbours
    for r in range(R):
        nb = [s for s in range(R) if oracle.mp_near(r, s, GRID)]
        assert len(out["children_at"][r]) == sum(int((nodes[s, 1:, 4] > 0).sum()) for s in nb)
    # node items carry the node exactly
    it = out["roots_at"][0][0]
    s = int(it[9])
    np.testing.assert_array_equal(it[:8].view(np.uint64), nodes[s, 0, :4])
    assert it[8] == nodes[s, 0, 4] and it[10] == oracle.MP_ROOT_CODE
