"""Pins for the oracle's streamline tracer (Sec. 5.4, RK4 on a trilinear field).

What fixes it independently of the oracle's own code:
  * trilinear sampling of a linear field is exact in the interior, and RK4 on
    a rotation field follows the exact rotation to O(h^5) per step, while a
    wrong stage or weight errs at O(h^2)..O(h^4);
  * a constant field gives straight lines: after k steps p = p0 + k h v;
  * the generated field is the curl of the stated potential: it matches the
    analytic curl at voxel centres and its discrete divergence is ~0;
  * termination rules: zero field stalls at once, maxSteps caps the steps,
    leaving the grid stops the particle just outside it.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_30294_gb300 import inputs


def _rotation_field(n, omega):
    c = n / 2.0
    ax = np.arange(n, dtype=np.float64) + 0.5
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    f = np.zeros((n, n, n, 3), np.float64)
    f[..., 0] = -omega * (y - c)
    f[..., 1] = omega * (x - c)
    return f.astype(np.float32)


def test_trilinear_velocity_of_linear_field_is_exact():
    n = 32
    f = _rotation_field(n, 0.05)
    rng = np.random.default_rng(1)
    for p in rng.uniform(1.0, n - 1.0, size=(50, 3)).astype(np.float32):
        v = oracle.c2_velocity(f, p)
        want = np.array([-0.05 * (p[1] - 16.0), 0.05 * (p[0] - 16.0), 0.0])
        np.testing.assert_allclose(v, want, atol=2e-6)


def test_rk4_step_follows_exact_rotation():
    n, omega, h = 64, 0.02, 0.25
    f = _rotation_field(n, omega)
    p0 = np.array([40.0, 32.0, 10.0], np.float32)
    q = oracle.c2_rk4(f, p0, h)
    ang = omega * h
    r = np.array([p0[0] - 32.0, p0[1] - 32.0])
    want = np.array([32.0 + math.cos(ang) * r[0] - math.sin(ang) * r[1],
                     32.0 + math.sin(ang) * r[0] + math.cos(ang) * r[1], p0[2]])
    err = np.abs(q - want).max()
    assert err < 1e-5
    # forward Euler (one stage) would miss by ~|r| (omega h)^2 / 2 = 5e-5 here
    euler = p0 + h * oracle.c2_velocity(f, p0)
    assert np.abs(euler - want).max() > 5 * err


def test_many_steps_stay_on_the_circle():
    n, omega = 64, 0.02
    f = _rotation_field(n, omega)
    seeds = np.array([[44.0, 32.0, 5.0]], np.float32)
    res = oracle.c2_trace(f, seeds, brick=16, h=0.25, max_steps=400)
    assert res["status"][0] == oracle.MAXSTEPS and res["steps"][0] == 400
    ang = omega * 0.25 * 400
    want = np.array([32.0 + 12.0 * math.cos(ang), 32.0 + 12.0 * math.sin(ang), 5.0])
    assert np.abs(res["pos"][0] - want).max() < 1e-3
    # 2 radians on the circle of radius 12 about (32, 32), counter-clockwise from
    # angle 0: y stays in [32, 48) and x crosses the brick face x = 32 once
    assert res["hops"][0] == 1


def test_constant_field_gives_straight_lines_and_exit():
    n = 32
    v = np.array([0.5, 0.25, -0.125], np.float32)
    f = np.broadcast_to(v, (n, n, n, 3)).astype(np.float32)
    seeds = np.array([[3.2, 7.7, 30.1]], np.float32)
    res = oracle.c2_trace(f, seeds, brick=8, h=0.25, max_steps=100000)
    k = int(res["steps"][0])
    assert res["status"][0] == oracle.EXITED
    # the particle leaves when x crosses 32: k = first step with 3.2 + 0.125 k >= 32
    assert k == math.ceil((32.0 - 3.2) / 0.125) or k == math.ceil((32.0 - 3.2) / 0.125) + 1
    np.testing.assert_allclose(res["pos"][0], seeds[0] + k * 0.25 * v, atol=2e-4)
    # bricks of 8: x crosses 8, 16, 24 (3 faces), y crosses 8 and 16 (7.7 -> 7.7 + 0.0625 k), z crosses 24
    y_end = 7.7 + 0.0625 * k
    z_end = 30.1 - 0.03125 * k
    want = 3 + sum(1 for b in (8, 16, 24) if 7.7 < b <= y_end) + sum(1 for b in (8, 16, 24) if z_end < b <= 30.1)
    assert res["hops"][0] == want


def test_stall_and_step_limit():
    n = 16
    f = np.zeros((n, n, n, 3), np.float32)
    res = oracle.c2_trace(f, np.array([[5.0, 5.0, 5.0]], np.float32), brick=8)
    assert res["status"][0] == oracle.STALLED and res["steps"][0] == 0
    np.testing.assert_array_equal(res["pos"][0], [5.0, 5.0, 5.0])
    f = _rotation_field(n, 0.01)
    res = oracle.c2_trace(f, np.array([[10.0, 8.0, 8.0]], np.float32), brick=8, max_steps=7)
    assert res["status"][0] == oracle.MAXSTEPS and res["steps"][0] == 7


def test_generated_field_is_the_curl_and_divergence_free():
    n = 32
    modes = inputs.c2_modes()
    f, scale = inputs.c2_field(n, modes=modes)
    rng = np.random.default_rng(3)
    idx = rng.integers(0, n, size=(40, 3))
    pts = idx.astype(np.float64) + 0.5
    want = inputs.c2_velocity_exact(pts, n, modes=modes, scale=scale)
    got = f[idx[:, 2], idx[:, 1], idx[:, 0]]
    np.testing.assert_allclose(got, want, atol=1e-6)
    assert abs(np.sqrt((f.astype(np.float64) ** 2).sum(-1)).max() - 1.0) < 1e-6


def _div_and_grad(d):
    div = ((d[1:-1, 1:-1, 2:, 0] - d[1:-1, 1:-1, :-2, 0]) + (d[1:-1, 2:, 1:-1, 1] - d[1:-1, :-2, 1:-1, 1])
           + (d[2:, 1:-1, 1:-1, 2] - d[:-2, 1:-1, 1:-1, 2])) / 2.0
    grad = np.abs(d[1:-1, 1:-1, 2:, 0] - d[1:-1, 1:-1, :-2, 0]).mean() / 2.0
    return np.abs(div).mean(), grad


def test_generated_field_is_divergence_free():
    # on a grid fine enough for the highest wavenumber (>= 16 cells per wave),
    # the central-difference divergence is only the truncation error, while a
    # field with the same modes but not a curl (a_m along k_m) is not
    n = 128
    k, a, phi = inputs.c2_modes()
    f, _ = inputs.c2_field(n, modes=(k, a, phi))
    div, grad = _div_and_grad(f.astype(np.float64))
    assert div < 0.1 * grad
    kh = k / np.linalg.norm(k, axis=1)[:, None]
    ax = np.arange(n, dtype=np.float64) + 0.5
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    pts = np.stack([x, y, z], -1)[::2, ::2, ::2]
    th = 2.0 * math.pi * (pts @ k.T) / n + phi
    ctrl = np.cos(th) @ kh  # longitudinal modes: divergence ~ |k|
    cd, cg = _div_and_grad(ctrl)
    assert cd > 0.5 * cg


def test_modes_recipe():
    k, a, phi = inputs.c2_modes()
    nk = np.linalg.norm(k, axis=1)
    assert k.shape == (32, 3) and np.all((nk >= 1) & (nk <= 8))
    assert np.all(k == np.round(k))
    assert np.abs((k * a).sum(1)).max() < 1e-12
    assert np.all((phi >= 0) & (phi < 2 * math.pi))


def test_seed_sets():
    sizes = inputs.c2_seed_set_sizes()
    assert sizes[0] == 4096 and sizes[-1] == 1 << 20 and sum(sizes) == 3383813
    s = inputs.c2_seeds(10000, 512)
    assert s.dtype == np.float32 and np.all(s >= 0) and np.all(s < 512)
