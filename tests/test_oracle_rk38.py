"""Pins of the oracle's fixed-step scheme (reading R18: Kutta's 3/8-rule RK4,
Sec. 2.3; the per-line step of Sec. 4 Eq. step).

- order: on B = (x, -y, 1) the footpoint error falls 16-fold per halving of the
  step (a wrong tableau entry breaks the fourth order);
- step counts worked out by hand on straight lines: each trial moves exactly
  the line's step, which is max(step_perp |Bn0/B|, step_min) (Eq. step);
- small steps converge to the RKF45 footpoints and Q.
"""
import math

import numpy as np

import oracle
import synth

G1 = synth.ANALYTIC_GRID
E2 = math.e ** 2 + math.e ** -2


def test_fourth_order_convergence():
    B = synth.analytic_cube("hyperbolic")
    seeds = np.array([[0.2, -0.1, 0.0], [-0.25, 0.3, 0.0], [0.1, 0.1, 0.0]])
    errs = []
    for step in (0.8, 0.4, 0.2):
        out = oracle.twist(B, G1, seeds, oracle.params(scheme=1, step=step))
        exact = np.stack([seeds[:, 0] * math.e, seeds[:, 1] / math.e, np.ones(3)], 1)
        assert np.all(out["face2"] == 5)
        errs.append(np.abs(out["r2"] - exact).max())
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    assert all(12.0 < r < 20.0 for r in ratios), (errs, ratios)


def _straight_count(length, h):
    # trials: floor(L/h) steps inside, the trial that leaves, the exit step
    return int(math.floor(length / h)) + 2


def test_uniform_field_step_count():
    # B = (0, 0, 1): a line from z = 0 runs 63 cells to the top; the backward
    # direction leaves through the seed's face at once (one trial and a
    # zero-length exit step)
    B = synth.analytic_cube("uniform")
    out = oracle.twist(B, G1, [[0.1, -0.3, 0.0]], oracle.params(scheme=1, step=0.4))
    assert int(out["steps"][0]) == _straight_count(63.0, 0.4) + 2
    np.testing.assert_allclose(out["r2"][0], [0.1, -0.3, 1.0], rtol=0, atol=1e-14)
    np.testing.assert_allclose(out["length"][0], 1.0, rtol=1e-14)


def test_eq_step_sets_the_line_step():
    # B = (1, 0, 3) on the z = 0 plane: |Bn0/B| = 3/sqrt(10), so the line steps
    # 3.0 x 0.9487 cells along a straight index-space path to the top
    B = np.ascontiguousarray(np.broadcast_to(np.array([1.0, 0.0, 3.0]), G1.shape))
    dx, dy, dz = G1.spacing
    bt = np.array([1.0 / dx, 0.0, 3.0 / dz])
    L = 63.0 * np.linalg.norm(bt) / bt[2]  # index-space length from z = 0 to the top
    plane = ((-0.9, -0.05, 0.0), (0.1, 0, 0), (0, 0.1, 0), 1, 1)
    for step, step_min in ((3.0, 0.15), (3.0, 2.9), (1.7, 0.15)):
        out = oracle.plane(B, G1, *plane, oracle.params(scheme=1, step=step, step_min=step_min))
        h = max(step * 3.0 / math.sqrt(10.0), step_min)
        assert out["face2"][0] == 5
        assert int(out["steps"][0]) == _straight_count(L, h) + 2, (step, step_min, out["steps"][0])


def test_small_steps_converge_to_rkf45():
    grid = synth.Grid((40, 36, 24), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    ch = synth.random_charges(np.random.default_rng(4), 6, ((0.0, 39.0), (0.0, 35.0)), depth=(6.0, 12.0))
    B = synth.monopole_cube(grid, ch, dtype=np.float64)
    plane = ((10.0, 8.0, 0.0), (0.5, 0, 0), (0, 0.5, 0), 16, 16)
    ref = oracle.plane(B, grid, *plane, oracle.params(tol=1e-11, max_steps=10 ** 7))
    fx = oracle.plane(B, grid, *plane, oracle.params(scheme=1, step=0.05, step_min=0.01, max_steps=10 ** 7))
    ok = np.isfinite(ref["Q"]) & np.isfinite(fx["Q"])
    assert ok.sum() > 200 and np.array_equal(ref["face2"], fx["face2"])
    # (a fixed step crossing a cell face, where the trilinear field's
    # derivative jumps, is locally second order: the agreement is 1e-6, not h^4)
    assert np.median(np.abs(fx["Q"][ok] / ref["Q"][ok] - 1)) < 1e-5
    assert np.abs(fx["r2"] - ref["r2"]).max() < 1e-4
    np.testing.assert_allclose(fx["Tw"], ref["Tw"], rtol=1e-5, atol=1e-8)
