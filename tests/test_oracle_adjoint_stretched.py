"""Pins of the adjoint oracle on stretched grids (reading R16: physical
positions, Eq. w0 weights in physical coordinates, each step scaled by the
widths of the cell it starts in, three-point curl stencils of a non-uniform
axis). The derivative is that of the traced computation with the step
sequence frozen (reading R13). Pinned by the C oracle's own stretched-grid map,
an exact invariance, a closed form and central differences of free re-traces."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
adj = pytest.importorskip("oracle.adjoint")

N = (24, 22, 16)
HI = (N[0] - 1.0, N[1] - 1.0, N[2] - 1.0)
Z0 = ((0.0, 0.0, 0.0), (HI[0] / 12, 0.0, 0.0), (0.0, HI[1] / 12, 0.0), 12, 12)
# an interior xz plane: seeds where |By/B| < 0.05 rotate S0
XZ = ((0.0, HI[1] * 0.41, 0.0), (HI[0] / 14, 0.0, 0.0), (0.0, 0.0, HI[2] / 9), 14, 9)


@pytest.fixture(scope="module")
def mono():
    grid = synth.stretched_grid(N, (0.0, 0.0, 0.0), HI, (1.03, 1.02, 1.05))
    ch = synth.random_charges(np.random.default_rng(5), 6, ((0.0, HI[0]), (0.0, HI[1])), depth=(2.0, 5.0))
    return synth.monopole_cube(grid, ch, dtype=np.float64), grid


def test_curl_matches_the_c_oracle(mono):
    B, grid = mono
    Jc = oracle.curl(B, grid)
    Jt = adj.curl_t_rect(torch.tensor(B), grid.coords).numpy()
    assert np.abs(Jt - Jc).max() <= 1e-14 * np.abs(Jc).max()


@pytest.mark.parametrize("plane", [Z0, XZ], ids=["z0_plane", "interior_xz_plane"])
def test_replay_reproduces_the_c_oracle(mono, plane):
    B, grid = mono
    p = oracle.params()
    ref = oracle.plane(B, grid, *plane, p)
    log = adj.lattice_log(B, grid, *plane, p)
    Q, Tw, usable, _ = adj.qmap_t(torch.tensor(B), grid, *plane, log)
    us = usable.numpy()
    assert us.sum() > 90
    np.testing.assert_allclose(Q.numpy()[us], ref["Q"][us], rtol=1e-11)
    np.testing.assert_allclose(Tw.numpy()[us], ref["Tw"][us], rtol=0, atol=1e-12)
    if plane is XZ:
        assert ((ref["status"][us] & oracle.ROTATED) != 0).sum() >= 5


@pytest.mark.parametrize("plane", [Z0, XZ], ids=["z0_plane", "interior_xz_plane"])
def test_gradient_orthogonal_to_B(mono, plane):
    # B -> c B leaves the frozen-sequence map unchanged, so <J^T w, B> = 0
    B, grid = mono
    m = plane[3] * plane[4]
    rng = np.random.default_rng(6)
    g, _ = adj.vjp(B, grid, *plane, rng.standard_normal(m), rng.standard_normal(m), oracle.params())
    assert np.linalg.norm(g) > 0
    assert abs(np.sum(g * B)) < 1e-12 * np.linalg.norm(g) * np.linalg.norm(B)


def test_hyperbolic_closed_form():
    # B = (a x, -a y, 1) on a stretched grid over [-1, 1]^2 x [0, 1]: Q = e^2a +
    # e^-2a on top exits, so dQ/da = 2 (e^2 - e^-2) at a = 1 along dB = (x, -y, 0)
    # (linear, so interpolated exactly on any grid); curl B = 0 stays 0
    grid = synth.stretched_grid((33, 33, 17), (-1.0, -1.0, 0.0), (1.0, 1.0, 1.0), (1.04, 1.04, 1.06))
    B = synth.analytic_cube("hyperbolic", grid)
    x, y, z = (np.asarray(c) for c in grid.coords)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    dB = np.stack([X, -Y, 0 * X], -1)
    plane = ((-0.3, -0.3, 0.0), (0.1, 0.0, 0.0), (0.0, 0.1, 0.0), 6, 6)
    p = oracle.params(tol=1e-10)
    w = np.random.default_rng(3).uniform(0.5, 1.5, 36)
    g, log = adj.vjp(B, grid, *plane, w, 0 * w, p)
    dQ, dTw, usable, _ = adj.jvp(B, grid, *plane, dB, p, log=log)
    assert usable.all()
    closed = 2.0 * (math.exp(2.0) - math.exp(-2.0))
    np.testing.assert_allclose(dQ, closed, rtol=1e-6)
    np.testing.assert_allclose(np.sum(g * dB), np.sum(w) * closed, rtol=1e-6)
    assert np.abs(dTw).max() < 1e-9


def test_gradient_matches_free_retrace_differences(mono):
    # central differences of free re-traces (steps chosen afresh) at tol 1e-8,
    # over the unperturbed map's usable seeds (the bounds of the uniform pin)
    B, grid = mono
    Bt = B * (1.0 + 0.05 * np.random.default_rng(8).standard_normal(B.shape))
    p = oracle.params(tol=1e-8, max_steps=1000000)
    tgt = oracle.plane(Bt, grid, *Z0, p)
    _, g, info = adj.loss_grad(B, grid, *Z0, tgt["Q"], tgt["Tw"], p, wtw=0.1)
    flat = np.abs(g).ravel()
    cand = np.nonzero(flat > 1e-2 * flat.max())[0]
    pick = np.random.default_rng(7).choice(cand, min(40, len(cand)), replace=False)
    eps = 1e-3 * float(np.sqrt(np.mean(B * B)))
    err = []
    for k in pick:
        Bp, Bm = B.copy().ravel(), B.copy().ravel()
        Bp[k] += eps
        Bm[k] -= eps
        lp = adj.free_loss(Bp.reshape(B.shape), grid, *Z0, tgt["Q"], tgt["Tw"], info["use"], p, 0.1)
        lm = adj.free_loss(Bm.reshape(B.shape), grid, *Z0, tgt["Q"], tgt["Tw"], info["use"], p, 0.1)
        err.append((lp - lm) / (2 * eps) - g.ravel()[k])
    err = np.abs(np.array(err))
    assert err.max() < 1e-2 * flat.max()
    assert np.median(err / flat[pick]) < 1e-2


@pytest.mark.parametrize("plane", [Z0, XZ], ids=["z0_plane", "interior_xz_plane"])
def test_fixed_step_replay_and_invariance(mono, plane):
    # the fixed-step 3/8 rule on the stretched grid (steps in cells of each
    # trial's start cell): the replay reproduces the C oracle's map, and the
    # frozen-sequence gradient is orthogonal to B
    B, grid = mono
    p = oracle.params(scheme=1, step=0.3, step_min=0.05, max_steps=10 ** 6)
    ref = oracle.plane(B, grid, *plane, p)
    log = adj.lattice_log(B, grid, *plane, p)
    Q, Tw, usable, _ = adj.qmap_t(torch.tensor(B), grid, *plane, log)
    us = usable.numpy()
    assert us.sum() > 90
    np.testing.assert_allclose(Q.numpy()[us], ref["Q"][us], rtol=1e-11)
    np.testing.assert_allclose(Tw.numpy()[us], ref["Tw"][us], rtol=0, atol=1e-12)
    m = plane[3] * plane[4]
    rng = np.random.default_rng(9)
    g, _ = adj.vjp(B, grid, *plane, rng.standard_normal(m), rng.standard_normal(m), p, log=log)
    assert np.linalg.norm(g) > 0
    assert abs(np.sum(g * B)) < 1e-12 * np.linalg.norm(g) * np.linalg.norm(B)
