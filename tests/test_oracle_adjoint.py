"""Pins of the FP64 CPU adjoint oracle (oracle/adjoint.py): the frozen-step
replay against the C oracle's own forward, and its derivatives against closed
forms, an exact invariance and finite differences of free re-traces.

The derivative is that of the map B -> (Q, Tw) with each line's accepted step
sizes, exit faces and exit kinds frozen at the values of the traced forward
(the discrete adjoint of the traced computation)."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
adj = pytest.importorskip("oracle.adjoint")

# the differentiation workload at 24^3 (tube radius and source depths scaled)
SMALL = dict(n=(24, 24, 24), count=6, radius_cells=4.0, dtype=np.float64)
PLANE16 = ((0.0, 0.0, 0.0), (23.0 / 16, 0.0, 0.0), (0.0, 23.0 / 16, 0.0), 16, 16)
PLANE8 = ((0.0, 0.0, 0.0), (23.0 / 8, 0.0, 0.0), (0.0, 23.0 / 8, 0.0), 8, 8)
# a 6x6 patch of the analytic grid's z=0 plane around the axis (every line leaves
# through the top for the hyperbolic and rotation fields)
PATCH = ((-0.3, -0.3, 0.0), (0.1, 0.0, 0.0), (0.0, 0.1, 0.0), 6, 6)


@pytest.fixture(scope="module")
def small():
    B, Bt, grid = synth.adjoint_cubes(**SMALL)
    return B, Bt, grid


def test_replay_reproduces_oracle_forward(small):
    B, _, grid = small
    p = oracle.params()
    ref = oracle.plane(B, grid, *PLANE16, p)
    log = adj.lattice_log(B, grid, *PLANE16, p)
    Q, Tw, usable, xi = adj.qmap_t(torch.tensor(B), grid, *PLANE16, log)
    us = usable.numpy()
    assert us.sum() > 200
    np.testing.assert_allclose(Q.numpy()[us], ref["Q"][us], rtol=1e-11)
    np.testing.assert_allclose(Tw.numpy()[us], ref["Tw"][us], rtol=0, atol=1e-12)
    r = np.asarray(grid.origin) + np.asarray(grid.spacing) * xi.numpy()
    np.testing.assert_allclose(r[us, 0], ref["r1"][us], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r[us, 1], ref["r2"][us], rtol=0, atol=1e-12)
    # faces and statuses are the oracle's
    assert np.array_equal(log["faces"][:, 0], ref["face1"]) and np.array_equal(log["faces"][:, 1], ref["face2"])


def test_gradient_orthogonal_to_B(small):
    # B -> c B leaves every line, Bn1 Bn2 / Bn0^2 and (J.B)/B^2 dl unchanged,
    # so the frozen-step map is exactly scale invariant: <dL/dB, B> = 0.
    B, Bt, grid = small
    p = oracle.params()
    tgt = oracle.plane(Bt, grid, *PLANE16, p)
    loss, g, _ = adj.loss_grad(B, grid, *PLANE16, tgt["Q"], tgt["Tw"], p)
    assert loss > 0 and np.linalg.norm(g) > 0
    assert abs(np.sum(g * B)) < 1e-12 * np.linalg.norm(g) * np.linalg.norm(B)


def _fd_check(B, Bt, grid, plane, wtw, picks, eps_rel):
    p = oracle.params(tol=1e-8, max_steps=1000000)
    tgt = oracle.plane(Bt, grid, *plane, p)
    _, g, info = adj.loss_grad(B, grid, *plane, tgt["Q"], tgt["Tw"], p, wtw=wtw)
    use = info["use"]
    flat = np.abs(g).ravel()
    cand = np.nonzero(flat > 1e-2 * flat.max())[0]
    rng = np.random.default_rng(7)
    pick = rng.choice(cand, min(picks, len(cand)), replace=False)
    eps = eps_rel * float(np.sqrt(np.mean(B * B)))
    err = []
    for k in pick:
        Bp = B.copy().ravel()
        Bm = B.copy().ravel()
        Bp[k] += eps
        Bm[k] -= eps
        lp = adj.free_loss(Bp.reshape(B.shape), grid, *plane, tgt["Q"], tgt["Tw"], use, p, wtw)
        lm = adj.free_loss(Bm.reshape(B.shape), grid, *plane, tgt["Q"], tgt["Tw"], use, p, wtw)
        err.append((lp - lm) / (2 * eps) - g.ravel()[k])
    err = np.abs(np.array(err))
    return err, g.ravel()[pick], flat.max()


def test_gradient_matches_free_retrace_fd(small):
    # Free re-traces choose their steps afresh, so their loss has small jumps
    # where an accept/reject decision flips and differs from the frozen map by
    # the step-size sensitivity; both shrink with the tolerance (1e-8 here).
    B, Bt, grid = small
    err, g, gmax = _fd_check(B, Bt, grid, PLANE8, 0.1, 64, 1e-3)
    assert err.max() < 1e-2 * gmax
    assert np.median(err / np.abs(g)) < 1e-2


def test_tw_gradient_matches_free_retrace_fd(small):
    # the Tw part alone (curl grid and the Tw integrand)
    B, Bt, grid = small
    err, g, gmax = _fd_check(B, Bt, grid, PLANE8, 1000.0, 48, 1e-3)
    assert err.max() < 1e-2 * gmax
    assert np.median(err / np.abs(g)) < 1e-2


def test_hyperbolic_field_closed_form():
    # B = (a x, -a y, 1): footpoints (x e^{aL}, y e^{-aL}) on top (L = 1), so
    # Q = e^{2aL} + e^{-2aL} and dQ/da = 2L (e^{2aL} - e^{-2aL}) along
    # dB = (x, -y, 0) (linear, hence exactly interpolated).
    grid = synth.ANALYTIC_GRID
    p = oracle.params()
    B = synth.analytic_cube("hyperbolic", grid)
    X, Y, Z = _mesh(grid)
    dB = np.stack([X, -Y, 0 * X], -1)
    m = PATCH[3] * PATCH[4]
    w = np.random.default_rng(3).uniform(0.5, 1.5, m)
    g, log = adj.vjp(B, grid, *PATCH, w, 0 * w, p)
    dQ, dTw, usable, _ = adj.jvp(B, grid, *PATCH, dB, p, log=log)
    assert usable.all()
    closed = 2.0 * (math.exp(2.0) - math.exp(-2.0))
    np.testing.assert_allclose(dQ, closed, rtol=1e-5)
    np.testing.assert_allclose(np.sum(g * dB), np.sum(w) * closed, rtol=1e-5)
    assert np.abs(dTw).max() < 1e-9  # curl B = 0 and stays 0 along dB


def test_rotation_field_closed_form():
    # B = (-q y, q x, 1): a line at radius r keeps it, J = (0, 0, 2q), so
    # Tw = q L / (2 pi sqrt(1 + q^2 r^2)) and dTw/dq = L (1 + q^2 r^2)^(-3/2) / (2 pi)
    # along dB = (-y, x, 0); the footpoint map stays a rotation (dQ/dq = 0).
    grid = synth.ANALYTIC_GRID
    q = 2.0 * math.pi
    p = oracle.params()
    B = synth.analytic_cube("rotation", grid, q=q)
    X, Y, Z = _mesh(grid)
    dB = np.stack([-Y, X, 0 * X], -1)
    m = PATCH[3] * PATCH[4]
    w = np.random.default_rng(4).uniform(0.5, 1.5, m)
    g, log = adj.vjp(B, grid, *PATCH, 0 * w, w, p)
    dQ, dTw, usable, _ = adj.jvp(B, grid, *PATCH, dB, p, log=log)
    assert usable.all()
    r0 = np.asarray(grid.origin) + np.asarray(grid.spacing) * adj.seeds_index(grid, *PATCH)
    r2 = r0[:, 0] ** 2 + r0[:, 1] ** 2
    closed = (1.0 + q * q * r2) ** -1.5 / (2.0 * math.pi)
    np.testing.assert_allclose(dTw, closed, rtol=1e-3)
    np.testing.assert_allclose(np.sum(g * dB), np.sum(w * closed), rtol=1e-3)
    assert np.abs(dQ).max() < 2e-3


def test_tangent_and_adjoint_modes_agree(small):
    # <J v, w> = <v, J^T w> between forward-mode and reverse-mode derivatives
    B, _, grid = small
    p = oracle.params()
    rng = np.random.default_rng(5)
    v = rng.standard_normal(B.shape)
    m = PLANE16[3] * PLANE16[4]
    wq, wt = rng.standard_normal(m), rng.standard_normal(m)
    g, log = adj.vjp(B, grid, *PLANE16, wq, wt, p)
    dQ, dTw, us, _ = adj.jvp(B, grid, *PLANE16, v, p, log=log)
    good = (log["status"] & oracle.BAD) == 0
    lhs = np.sum(wq[us] * dQ[us]) + np.sum(wt[good] * dTw[good])
    rhs = np.sum(v * g)
    assert abs(lhs - rhs) < 1e-11 * (abs(lhs) + np.linalg.norm(g) * np.linalg.norm(v) * 1e-3)


def _mesh(grid):
    x, y, z = (grid.axis(a) for a in range(3))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


# an interior xz plane of the 24^3 case: 21 seeds rotate S0
XZ = ((0.0, 18.3, 0.0), (23.0 / 20, 0.0, 0.0), (0.0, 0.0, 23.0 / 12), 20, 12)


def test_replay_of_rotated_seeds_reproduces_oracle(small):
    # a rotated seed's Q comes from its four extra lines, whose seeds the
    # replay places with the frame of B at the seed
    B, _, grid = small
    p = oracle.params()
    ref = oracle.plane(B, grid, *XZ, p)
    log = adj.lattice_log(B, grid, *XZ, p)
    Q, Tw, usable, _ = adj.qmap_t(torch.tensor(B), grid, *XZ, log)
    us = usable.numpy()
    rot = (ref["status"] & oracle.ROTATED) != 0
    assert (us & rot).sum() >= 15
    np.testing.assert_allclose(Q.numpy()[us], ref["Q"][us], rtol=1e-11)
    assert np.array_equal(us, np.isfinite(ref["Q"]))


def test_rotated_seed_gradient_at_its_cell(small):
    # the frame's dependence on B enters through the 8 nodes of the seed's
    # cell: central differences of free re-traces (tol 1e-9) on those 24
    # entries (a frame held constant misses by about 9 %)
    B, _, grid = small
    pt = oracle.params(tol=1e-9, max_steps=1000000)
    ref = oracle.plane(B, grid, *XZ, pt)
    rot = np.nonzero(((ref["status"] & oracle.ROTATED) != 0) & np.isfinite(ref["Q"]))[0]
    s = rot[len(rot) // 2]
    m = XZ[3] * XZ[4]
    w = np.zeros(m)
    w[s] = 1.0 / ref["Q"][s]
    c = np.floor(adj.seeds_index(grid, *XZ)[s]).astype(int)
    nx, ny, _ = grid.n
    ents = [(((c[2] + dz) * ny + (c[1] + dy)) * nx + (c[0] + dx)) * 3 + comp
            for dz in (0, 1) for dy in (0, 1) for dx in (0, 1) for comp in range(3)]
    eps = 1e-4 * float(np.sqrt(np.mean(B * B)))
    fd = []
    for k in ents:
        Bp = B.copy().ravel()
        Bm = B.copy().ravel()
        Bp[k] += eps
        Bm[k] -= eps
        qp = oracle.plane(Bp.reshape(B.shape), grid, *XZ, pt)["Q"][s]
        qm = oracle.plane(Bm.reshape(B.shape), grid, *XZ, pt)["Q"][s]
        fd.append(w[s] * (qp - qm) / (2 * eps))
    fd = np.array(fd)
    g, _ = adj.vjp(B, grid, *XZ, w, 0 * w, pt)
    assert np.linalg.norm(g.ravel()[ents] - fd) < 3e-2 * np.linalg.norm(fd)
    assert abs(np.sum(g * B)) < 1e-12 * np.linalg.norm(g) * np.linalg.norm(B)


def test_fixed_step_scheme_replay_and_gradient(small):
    # the 3/8-rule scheme (reading R18): the replay reproduces the C oracle's
    # map, the frozen-sequence map stays scale invariant, and at a small step
    # (where the step's own dependence on B through |Bn0/B| moves the map by
    # the integration error only) the gradient matches central differences of
    # free re-traces
    B, Bt, grid = small
    p = oracle.params(scheme=1, step=0.3, step_min=0.05, max_steps=10 ** 6)
    ref = oracle.plane(B, grid, *PLANE16, p)
    log = adj.lattice_log(B, grid, *PLANE16, p)
    assert log["scheme"] == 1
    Q, Tw, usable, _ = adj.qmap_t(torch.tensor(B), grid, *PLANE16, log)
    us = usable.numpy()
    assert us.sum() > 200
    np.testing.assert_allclose(Q.numpy()[us], ref["Q"][us], rtol=1e-11)
    np.testing.assert_allclose(Tw.numpy()[us], ref["Tw"][us], rtol=0, atol=1e-12)
    tgt = oracle.plane(Bt, grid, *PLANE8, p)
    loss, g, info = adj.loss_grad(B, grid, *PLANE8, tgt["Q"], tgt["Tw"], p, wtw=0.1)
    assert abs(np.sum(g * B)) < 1e-12 * np.linalg.norm(g) * np.linalg.norm(B)
    flat = np.abs(g).ravel()
    cand = np.nonzero(flat > 1e-2 * flat.max())[0]
    pick = np.random.default_rng(8).choice(cand, min(48, len(cand)), replace=False)
    eps = 1e-3 * float(np.sqrt(np.mean(B * B)))
    err = []
    for k in pick:
        Bp = B.copy().ravel()
        Bm = B.copy().ravel()
        Bp[k] += eps
        Bm[k] -= eps
        lp = adj.free_loss(Bp.reshape(B.shape), grid, *PLANE8, tgt["Q"], tgt["Tw"], info["use"], p, 0.1)
        lm = adj.free_loss(Bm.reshape(B.shape), grid, *PLANE8, tgt["Q"], tgt["Tw"], info["use"], p, 0.1)
        err.append((lp - lm) / (2 * eps) - g.ravel()[k])
    err = np.abs(np.array(err))
    # (measured: median relative error 2e-7, largest 2.6e-3 of the largest
    # entry, from entries at seed cells where the step's |Bn0/B| moves)
    assert err.max() < 1e-2 * flat.max()
    assert np.median(err / np.abs(g.ravel()[pick])) < 1e-5
