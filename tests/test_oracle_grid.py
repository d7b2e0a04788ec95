"""Pins of the oracle's grid operations against definitions that do not come
from the oracle itself: trilinear interpolation (Sec. 2.2, Eqs. interp, w0,
w1), the curl grid used by Eq. tw, and the gradient grid of B/|B|
(Eq. grad_B)."""
import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

import oracle
import synth


def _trilinear_poly(c, x, y, z):
    return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * y + c[5] * y * z + c[6] * x * z
            + c[7] * x * y * z)


def test_interp_reproduces_trilinear_polynomials(oracle_lib):
    rng = np.random.default_rng(1)
    n = (5, 4, 6)
    c = rng.standard_normal((3, 8))
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    arr = np.stack([_trilinear_poly(c[m], i, j, k) for m in range(3)], axis=-1)
    xi = rng.uniform([0, 0, 0], [n[0] - 1, n[1] - 1, n[2] - 1], size=(200, 3))
    got = oracle.interp(arr, n, xi)
    # within one cell a trilinear polynomial is reproduced exactly
    cell = np.floor(xi)
    ok = np.all(cell < np.array(n) - 1, axis=1)
    want = np.stack([_trilinear_poly(c[m], xi[:, 0], xi[:, 1], xi[:, 2]) for m in range(3)], axis=1)
    # a global trilinear polynomial is trilinear in every cell
    assert np.max(np.abs(got[ok] - want[ok])) < 1e-12


def test_interp_matches_scipy_linear_on_random_nodes(oracle_lib):
    rng = np.random.default_rng(2)
    n = (7, 5, 6)
    arr = rng.standard_normal((n[2], n[1], n[0], 2))
    xi = rng.uniform(0, 1, size=(300, 3)) * (np.array(n) - 1)
    got = oracle.interp(arr, n, xi)
    for m in range(2):
        f = RegularGridInterpolator((np.arange(n[2]), np.arange(n[1]), np.arange(n[0])), arr[..., m])
        want = f(xi[:, ::-1])
        assert np.max(np.abs(got[:, m] - want)) < 1e-13


def test_interp_nodes_and_extrapolation(oracle_lib):
    rng = np.random.default_rng(3)
    n = (4, 4, 4)
    arr = rng.standard_normal((4, 4, 4, 1))
    idx = np.array([[0, 0, 0], [3, 3, 3], [1, 2, 3], [3, 0, 2]], dtype=float)
    got = oracle.interp(arr, n, idx)[:, 0]
    want = arr[idx[:, 2].astype(int), idx[:, 1].astype(int), idx[:, 0].astype(int), 0]
    assert np.allclose(got, want, rtol=0, atol=1e-15)
    # outside the box the clamped boundary cell extrapolates linearly (reading R3)
    k, j, i = np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij")
    lin = (1.0 + 2.0 * i - 0.5 * j + 0.25 * k)[..., None]
    pts = np.array([[-0.5, 1.0, 1.0], [3.5, 2.0, -0.25], [1.0, 4.0, 3.2]])
    got = oracle.interp(lin, n, pts)[:, 0]
    want = 1.0 + 2.0 * pts[:, 0] - 0.5 * pts[:, 1] + 0.25 * pts[:, 2]
    assert np.allclose(got, want, rtol=0, atol=1e-13)


def _quadratic_field(grid, c):
    x, y, z = (grid.axis(a) for a in range(3))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    mons = [np.ones_like(X), X, Y, Z, X * X, Y * Y, Z * Z, X * Y, Y * Z, X * Z]
    B = np.stack([sum(c[m, t] * mons[t] for t in range(10)) for m in range(3)], axis=-1)
    return B, (X, Y, Z)


def _d_quadratic(c, X, Y, Z, axis):
    # derivative of the 10-term quadratic along axis
    if axis == 0:
        return c[1] + 2 * c[4] * X + c[7] * Y + c[9] * Z
    if axis == 1:
        return c[2] + 2 * c[5] * Y + c[7] * X + c[8] * Z
    return c[3] + 2 * c[6] * Z + c[8] * Y + c[9] * X


def test_curl_exact_for_quadratic_fields(oracle_lib):
    """Central and 2nd-order one-sided differences (reading R4) are exact for
    quadratics, so the curl grid equals the analytic curl at every node,
    faces and edges included."""
    rng = np.random.default_rng(4)
    grid = synth.Grid((6, 5, 7), (-0.3, 0.2, 0.0), (0.1, 0.2, 0.15))
    c = rng.standard_normal((3, 10))
    B, (X, Y, Z) = _quadratic_field(grid, c)
    J = oracle.curl(B, grid)
    d = lambda m, a: _d_quadratic(c[m], X, Y, Z, a)  # noqa: E731
    want = np.stack([d(2, 1) - d(1, 2), d(0, 2) - d(2, 0), d(1, 0) - d(0, 1)], axis=-1)
    assert np.max(np.abs(J - want)) < 1e-10


def test_curl_and_gradb_match_numpy_gradient(oracle_lib):
    rng = np.random.default_rng(5)
    B, grid = synth.random_smooth_cube(rng, n=(9, 8, 7))
    J = oracle.curl(B, grid)
    G = oracle.gradb(B, grid)
    dx, dy, dz = grid.spacing
    # np.gradient: 2nd-order central inside, 2nd-order one-sided at the edges
    g = [[np.gradient(B[..., m], dz, dy, dx, edge_order=2)[::-1][a] for a in range(3)] for m in range(3)]
    want = np.stack([g[2][1] - g[1][2], g[0][2] - g[2][0], g[1][0] - g[0][1]], axis=-1)
    assert np.max(np.abs(J - want)) < 1e-11
    bh = B / np.linalg.norm(B, axis=-1, keepdims=True)
    gb = [np.gradient(bh[..., b], dz, dy, dx, edge_order=2)[::-1] for b in range(3)]
    for a in range(3):
        for b in range(3):
            assert np.max(np.abs(G[..., 3 * a + b] - gb[b][a])) < 1e-11


def test_curl_two_node_axis_is_first_order(oracle_lib):
    grid = synth.Grid((2, 3, 3), (0.0, 0.0, 0.0), (0.5, 1.0, 1.0))
    x = grid.axis(0)
    k, j, i = np.meshgrid(np.arange(3), np.arange(3), np.arange(2), indexing="ij")
    B = np.zeros((3, 3, 2, 3))
    B[..., 1] = 3.0 * x[i]  # By = 3x  ->  Jz = 3
    J = oracle.curl(B, grid)
    assert np.allclose(J[..., 2], 3.0) and np.allclose(J[..., :2], 0.0)


def test_rejects_degenerate_grid(oracle_lib):
    grid = synth.Grid((1, 3, 3), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    with pytest.raises(ValueError):
        oracle.curl(np.zeros((3, 3, 1, 3)), grid)
