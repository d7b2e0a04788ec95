"""Pins of the oracle on stretched (rectilinear) grids, reading R16 (Sec. 2.2
Eqs. interp, w0, w1 with a cell search; Sec. 2.3 per-cell step and tolerance
scaling).

The pins come from outside the oracle: library routines (numpy's searchsorted
and second-order gradient on non-uniform axes, scipy's grid interpolator),
polynomials the stencils reproduce exactly, closed forms of linear fields
(exact under trilinear interpolation on any rectilinear grid), the uniform
grid as a special case, and the step sequence of a constant field worked out
by hand.
"""
import math

import numpy as np
import pytest

import oracle
import synth

E2 = math.e ** 2 + math.e ** -2
BOX = ((-1.0, -1.0, 0.0), (1.0, 1.0, 1.0))


def _grid(n=(40, 36, 30), ratios=(1.04, 1.05, 1.06)):
    return synth.stretched_grid(n, *BOX, ratios=ratios)


def test_stretched_axis_recipe():
    x = np.asarray(synth.stretched_axis(9, 0.0, 8.0, 1.1, "bottom"))
    w = np.diff(x)
    assert x[0] == 0.0 and x[-1] == 8.0 and np.all(w > 0)
    np.testing.assert_allclose(w[1:] / w[:-1], 1.1, rtol=1e-12)
    y = np.asarray(synth.stretched_axis(11, -1.0, 1.0, 1.2, "edges"))
    wy = np.diff(y)
    np.testing.assert_allclose(wy, wy[::-1], rtol=1e-12)
    assert wy[0] > wy[4]
    np.testing.assert_allclose(synth.stretched_axis(5, 0.0, 4.0, 1.0), [0, 1, 2, 3, 4], atol=1e-15)


def test_cell_search_matches_searchsorted():
    rng = np.random.default_rng(1)
    X = np.asarray(synth.stretched_axis(37, -2.0, 5.0, 1.07, "edges"))
    x = np.concatenate([rng.uniform(-3.0, 6.0, 2000), X, [-np.inf, np.inf, np.nan]])
    got = oracle.cell_rect(X, x)
    want = np.clip(np.searchsorted(X, x, side="right") - 1, 0, len(X) - 2)
    want[np.isnan(x)] = 0
    assert np.array_equal(got, want)


def test_interp_reproduces_trilinear_polynomials():
    g = _grid()
    x, y, z = (g.axis(a) for a in range(3))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    f = np.stack([1 + 2 * X - Y + 0.5 * Z, X * Y * Z - 3 * X * Z + 0.25, (1 - X) * (2 + Y) * (3 - Z)], -1)
    rng = np.random.default_rng(2)
    r = rng.uniform((-1, -1, 0), (1, 1, 1), (500, 3))
    got = oracle.interp_rect(f, g, r)
    X, Y, Z = r.T
    want = np.stack([1 + 2 * X - Y + 0.5 * Z, X * Y * Z - 3 * X * Z + 0.25, (1 - X) * (2 + Y) * (3 - Z)], -1)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def test_interp_matches_scipy_on_a_random_field():
    interp = pytest.importorskip("scipy.interpolate")
    g = _grid((17, 13, 11))
    rng = np.random.default_rng(3)
    f = rng.standard_normal(g.shape)
    r = rng.uniform((-1, -1, 0), (1, 1, 1), (400, 3))
    got = oracle.interp_rect(f, g, r)
    ref = interp.RegularGridInterpolator((g.axis(2), g.axis(1), g.axis(0)), f, method="linear")(r[:, ::-1])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


def test_curl_exact_for_quadratics_and_matches_numpy_gradient():
    g = _grid((15, 12, 10))
    x, y, z = (g.axis(a) for a in range(3))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    # each component quadratic in each coordinate: the three-point stencils are exact
    B = np.stack([Y * Y + 2 * Z * Z - X * Y, X * Z - 3 * Z * Z + X * X, X * X * Y + Y * Y - 2 * X], -1)
    J = oracle.curl(B, g)
    want = np.stack([(X * X + 2 * Y) - (X - 6 * Z), (4 * Z) - (2 * X * Y - 2), (Z + 2 * X) - (2 * Y - X)], -1)
    np.testing.assert_allclose(J, want, rtol=0, atol=1e-11)
    rng = np.random.default_rng(4)
    R = rng.standard_normal(g.shape)
    JR = oracle.curl(R, g)
    d = [np.gradient(R[..., c], z, y, x, edge_order=2) for c in range(3)]  # d[c][axis] with axis order z, y, x
    ref = np.stack([d[2][1] - d[1][0], d[0][0] - d[2][2], d[1][2] - d[0][1]], -1)
    np.testing.assert_allclose(JR, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def _seeds(nu=24, lo=-0.9, hi=0.9):
    d = (hi - lo) / nu
    return d, (lo, lo, 0.0), (d, 0.0, 0.0), (0.0, d, 0.0)


def test_hyperbolic_closed_form_on_a_stretched_grid():
    # B = (x, -y, 1): x = x0 e^z, y = y0 e^-z, Q = e^2 + e^-2 on top exits
    g = _grid()
    B = synth.analytic_cube("hyperbolic", g)
    d, o, u, v = _seeds(24, -0.3, 0.3)
    out = oracle.plane(B, g, o, u, v, 24, 24, oracle.params(tol=1e-10))
    xs = o[0] + (np.arange(24) + 0.5) * d
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    X, Y = X.ravel(), Y.ravel()
    assert np.all(out["status"] == 0) and np.all(out["face2"] == 5)
    np.testing.assert_allclose(out["r2"][:, 0], X * math.e, rtol=0, atol=1e-8)
    np.testing.assert_allclose(out["r2"][:, 1], Y / math.e, rtol=0, atol=1e-8)
    np.testing.assert_allclose(out["Q"], E2, rtol=1e-8)
    np.testing.assert_allclose(out["Tw"], 0.0, atol=1e-12)


def test_rotation_closed_form_on_a_stretched_grid():
    # B = (-q y, q x, 1): Q = 2, Tw = q L / (2 pi sqrt(1 + q^2 r^2)), L = 1
    q = 2.0 * math.pi
    g = _grid()
    B = synth.analytic_cube("rotation", g, q=q)
    d, o, u, v = _seeds(16, -0.25, 0.25)
    out = oracle.plane(B, g, o, u, v, 16, 16, oracle.params(tol=1e-10))
    xs = o[0] + (np.arange(16) + 0.5) * d
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    r2 = (X * X + Y * Y).ravel()
    assert np.all(out["status"] == 0)
    np.testing.assert_allclose(out["Tw"], q / (2 * math.pi * np.sqrt(1 + q * q * r2)), rtol=1e-7)
    np.testing.assert_allclose(out["Q"], 2.0, rtol=1e-6)
    np.testing.assert_allclose(out["length"], np.sqrt(1 + q * q * r2), rtol=1e-8)


def test_uniform_field_step_sequence():
    # B = (0, 0, 1) on a z axis with cells growing by 1.3: zero error, so h
    # grows x4 per step from h0 = 0.5 up to h_max = 4 (cells); each step moves
    # h times the width of the cell it starts in (R16) until the next step
    # would leave the box, then one exit step lands on the top face.
    zs = np.asarray(synth.stretched_axis(12, 0.0, 1.0, 1.3, "bottom"))
    g = synth.RectGrid((synth.stretched_axis(5, -1.0, 1.0, 1.0), synth.stretched_axis(5, -1.0, 1.0, 1.0),
                        tuple(zs)))
    B = synth.analytic_cube("uniform", g)
    p = oracle.params(tol=1e-6)
    out = oracle.twist(B, g, [[0.1, -0.2, 0.0]], p)
    z, h, trials = 0.0, p.h0, 0
    while True:
        c = min(np.searchsorted(zs, z, side="right") - 1, len(zs) - 2)
        zn = z + h * (zs[c + 1] - zs[c])
        trials += 1
        if zn > 1.0:
            trials += 1  # the exit step
            break
        z, h = zn, min(4.0 * h, p.hmax)
    # the backward direction leaves through the seed's own face at once:
    # one trial that exits and one zero-length exit step
    assert int(out["steps"][0]) == trials + 2
    assert out["face2"][0] == 5 and out["face1"][0] == 4
    np.testing.assert_allclose(out["r2"][0], [0.1, -0.2, 1.0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(out["length"][0], 1.0, rtol=1e-14)


def _monopole(grid):
    rng = np.random.default_rng(5)
    hi = grid.hi
    ch = synth.random_charges(rng, 8, ((grid.origin[0], hi[0]), (grid.origin[1], hi[1])), depth=(2.0, 6.0))
    return synth.monopole_cube(grid, ch, dtype=np.float64)


def test_uniform_coordinates_reduce_to_the_uniform_method():
    # a RectGrid whose coordinates are uniform (anisotropic spacing) gives the
    # method of R1-R2 in exact arithmetic; at a tight tolerance both agree to
    # the integration error
    ug = synth.Grid((21, 19, 13), (-3.0, -2.0, 0.0), (0.5, 0.5, 0.25))
    rg = synth.RectGrid(tuple(tuple(float(v) for v in ug.axis(a)) for a in range(3)))
    B = _monopole(ug)
    assert np.array_equal(B, _monopole(rg))
    plane = ((-3.0, -2.0, 0.0), (10.0 / 16, 0.0, 0.0), (0.0, 9.0 / 16, 0.0), 16, 16)
    p = oracle.params(tol=1e-10)
    a = oracle.plane(B, ug, *plane, p)
    b = oracle.plane(B, rg, *plane, p)
    assert np.array_equal(a["face1"], b["face1"]) and np.array_equal(a["face2"], b["face2"])
    assert np.array_equal(a["status"] & oracle.BAD, b["status"] & oracle.BAD)
    ok = np.isfinite(a["Q"])
    assert ok.sum() > 200
    # the two differ by rounding, which the adaptive steps carry into
    # differences of the order of the integration error (they shrink with
    # tol: medians 1.2e-7, 1.9e-9, 2.9e-11 at tol 1e-8, 1e-10, 1e-12)
    dr = np.abs(np.concatenate([b["r1"] - a["r1"], b["r2"] - a["r2"]])).max(1)
    assert np.median(dr) < 1e-8 and np.percentile(dr, 99) < 1e-6
    assert np.median(np.abs(b["Q"][ok] / a["Q"][ok] - 1)) < 1e-7
    assert np.median(np.abs(b["Tw"] - a["Tw"])) < 1e-9
    # the per-cell scaling of the error norm matters: at the default tolerance
    # the trial counts are the uniform method's (rounding aside)
    pd = oracle.params()
    sa = oracle.plane(B, ug, *plane, pd)["steps"]
    sb = oracle.plane(B, rg, *plane, pd)["steps"]
    assert np.mean(sa == sb) > 0.9


def test_line_invariants_on_a_stretched_grid():
    # Q >= 2 up to the finite-difference error, and a line traced again from
    # its own end footpoint has the same Tw and length
    g = _grid((33, 29, 21), (1.06, 1.06, 1.1))
    B = _monopole(g)
    p = oracle.params(tol=1e-9)
    d, o, u, v = _seeds(20, -0.3, 0.3)  # a lattice fine enough for the differences (0.03)
    out = oracle.plane(B, g, o, u, v, 20, 20, p)
    ok = np.isfinite(out["Q"])
    assert ok.sum() > 300
    assert out["Q"][ok].min() > 1.995
    good = (out["status"] & oracle.BAD) == 0
    sel = np.nonzero(good)[0][::7]
    again = oracle.twist(B, g, out["r2"][sel], p)
    np.testing.assert_allclose(again["Tw"], out["Tw"][sel], rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(again["length"], out["length"][sel], rtol=1e-6)


def test_gradb_grid_matches_numpy_gradient():
    # Method II way 1: d(B_b/|B|)/dx_a at the nodes with the same three-point
    # stencils as the curl
    g = _grid((15, 12, 10))
    rng = np.random.default_rng(6)
    B = rng.standard_normal(g.shape) + np.array([0.0, 0.0, 3.0])
    G = oracle.gradb(B, g)
    bh = B / np.linalg.norm(B, axis=-1, keepdims=True)
    x, y, z = (g.axis(a) for a in range(3))
    for b in range(3):
        dz, dy, dx = np.gradient(bh[..., b], z, y, x, edge_order=2)
        for a, d in enumerate((dx, dy, dz)):
            np.testing.assert_allclose(G[..., 3 * a + b], d, rtol=0, atol=1e-9 * np.abs(d).max())


def test_method2_closed_forms_on_a_stretched_grid():
    # deviation vectors (way 2) carry no finite-difference error of the
    # lattice: B = (x, -y, 1) gives Q = e^2 + e^-2 on top exits, and the rigid
    # rotation Q_perp = 2
    g = _grid()
    d, o, u, v = _seeds(12, -0.3, 0.3)
    B = synth.analytic_cube("hyperbolic", g)
    out = oracle.plane(B, g, o, u, v, 12, 12, oracle.params(method=2, way=2, tol=1e-10))
    assert np.all(out["face2"] == 5)
    np.testing.assert_allclose(out["Q"], E2, rtol=1e-6)
    B = synth.analytic_cube("rotation", g, q=2.0 * math.pi)
    out = oracle.plane(B, g, o, u, v, 12, 12, oracle.params(method=2, way=2, tol=1e-10, qperp=1))
    np.testing.assert_allclose(out["Q"], 2.0, rtol=1e-6)


def test_method2_uniform_coordinates_reduce_to_the_uniform_method():
    ug = synth.Grid((21, 19, 13), (-3.0, -2.0, 0.0), (0.5, 0.5, 0.25))
    rg = synth.RectGrid(tuple(tuple(float(v) for v in ug.axis(a)) for a in range(3)))
    B = _monopole(ug)
    plane = ((-3.0, -2.0, 0.0), (10.0 / 16, 0.0, 0.0), (0.0, 9.0 / 16, 0.0), 16, 16)
    # way 1 converges with the tolerance (median 1.6e-9 at 1e-10); way 2's
    # +-0.001-cell differences have kinks where a stage point comes within
    # 0.001 cells of a cell face, so two step sequences that differ by rounding
    # keep differences near 1e-5 at any tolerance
    for way, bound in ((1, 1e-7), (2, 1e-4)):
        p = oracle.params(method=2, way=way, tol=1e-10)
        a = oracle.plane(B, ug, *plane, p)
        b = oracle.plane(B, rg, *plane, p)
        ok = np.isfinite(a["Q"])
        assert ok.sum() > 200 and np.array_equal(a["face2"], b["face2"])
        assert np.median(np.abs(b["Q"][ok] / a["Q"][ok] - 1)) < bound


def test_fixed_step_scheme_on_a_stretched_grid():
    # B = (0, 0, 1) on a z axis with cells growing by 1.3 and the 3/8 rule:
    # every trial moves h times the width of the cell it starts in
    zs = np.asarray(synth.stretched_axis(12, 0.0, 1.0, 1.3, "bottom"))
    g = synth.RectGrid((synth.stretched_axis(5, -1.0, 1.0, 1.0), synth.stretched_axis(5, -1.0, 1.0, 1.0),
                        tuple(zs)))
    B = synth.analytic_cube("uniform", g)
    out = oracle.twist(B, g, [[0.1, -0.2, 0.0]], oracle.params(scheme=1, step=0.7))
    z, trials = 0.0, 0
    while True:
        c = min(np.searchsorted(zs, z, side="right") - 1, len(zs) - 2)
        zn = z + 0.7 * (zs[c + 1] - zs[c])
        trials += 1
        if zn > 1.0:
            trials += 1
            break
        z = zn
    assert int(out["steps"][0]) == trials + 2
    np.testing.assert_allclose(out["r2"][0], [0.1, -0.2, 1.0], rtol=0, atol=1e-15)
    # and the hyperbolic closed form at a small step
    g = _grid()
    d, o, u, v = _seeds(10, -0.3, 0.3)
    out = oracle.plane(synth.analytic_cube("hyperbolic", g), g, o, u, v, 10, 10,
                       oracle.params(scheme=1, step=0.1, step_min=0.01))
    assert np.all(out["face2"] == 5)
    np.testing.assert_allclose(out["Q"], E2, rtol=2e-5)
