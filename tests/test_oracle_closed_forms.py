"""Closed-form pins of the oracle's tracer and Q/Tw assembly on linear
divergence-free fields, where trilinear interpolation and the curl grid are
exact and every footpoint map is known analytically.

Q definitions: Eqs. D+-, Q+-, Bn1 (Sec. 1), Method I Eqs. D+-2/D+-3 and
Method II Eqs. rb2/q_scott (Sec. 2.1); Tw: Eq. tw (Sec. 1).
"""
import math

import numpy as np
import pytest

import oracle
import synth

G1 = synth.ANALYTIC_GRID
E2 = math.e ** 2 + math.e ** -2


def _lattice(nu=32):
    d = 2.0 / nu
    xs = -1.0 + (np.arange(nu) + 0.5) * d
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    return d, X.ravel(), Y.ravel()


def _plane(kind, z=0.0, nu=32, **kw):
    d, X, Y = _lattice(nu)
    B = synth.analytic_cube(kind)
    p = oracle.params(**{"tol": 1e-10, **kw})
    return oracle.plane(B, G1, (-1.0, -1.0, z), (d, 0, 0), (0, d, 0), nu, nu, p), X, Y, d


@pytest.mark.parametrize("method,way", [(1, 1), (2, 1), (2, 2)])
def test_uniform_field(oracle_lib, method, way):
    o, X, Y, _ = _plane("uniform", method=method, way=way)
    assert np.all(o["status"] == 0)
    assert np.all(o["face1"] == 4) and np.all(o["face2"] == 5)
    assert np.allclose(o["Q"], 2.0, rtol=1e-12)
    assert np.allclose(o["Tw"], 0.0, atol=1e-15)
    assert np.allclose(o["length"], 1.0, rtol=1e-12)
    assert np.allclose(o["r2"], np.stack([X, Y, np.ones_like(X)], 1), atol=1e-12)
    assert np.allclose(o["r1"], np.stack([X, Y, np.zeros_like(X)], 1), atol=0)


def test_hyperbolic_top_exits_method1(oracle_lib):
    """B=(x,-y,1): x = x0 e^z, y = y0 e^-z; top exits have Q = e^2 + e^-2."""
    o, X, Y, d = _plane("hyperbolic", nu=64)
    top = np.abs(X) < 1 / math.e - 2 * d
    assert top.sum() > 500
    assert np.all(o["face2"][top] == 5) and np.all(o["face1"][top] == 4)
    assert np.max(np.abs(o["r2"][top, 0] - X[top] * math.e)) < 1e-8
    assert np.max(np.abs(o["r2"][top, 1] - Y[top] / math.e)) < 1e-8
    assert np.max(np.abs(o["Q"][top] / E2 - 1)) < 1e-8


def test_hyperbolic_side_exits_method1(oracle_lib):
    """Side exits land on x = sign(x0) at (y, z) = (y0 |x0|, -ln|x0|); Method I
    must equal the same finite-difference stencil applied to those exact
    footpoints (reading R8)."""
    o, X, Y, d = _plane("hyperbolic", nu=64)
    side = np.abs(X) > 1 / math.e + 2 * d
    ax = np.abs(X)
    assert np.all(o["face2"][side] == np.where(X[side] > 0, 1, 0))
    assert np.max(np.abs(o["r2"][side, 1] - Y[side] * ax[side])) < 1e-8
    assert np.max(np.abs(o["r2"][side, 2] + np.log(ax[side]))) < 1e-8
    # exact footpoint map F(x0,y0) = (y0|x0|, -ln|x0|); central differences in x0 and y0
    F = lambda x, y: np.stack([y * np.abs(x), -np.log(np.abs(x))], -1)  # noqa: E731
    jx = (F(X + d, Y) - F(X - d, Y)) / (2 * d)
    jy = (F(X, Y + d) - F(X, Y - d)) / (2 * d)
    q_fd = (jx ** 2).sum(-1) + (jy ** 2).sum(-1)  # J1 = I, |Bn1 Bn2| / Bn0^2 = 1
    inner = side & (np.abs(Y) < 1 - 1.5 * d) & (np.abs(X) < 1 - 1.5 * d)
    assert np.max(np.abs(o["Q"][inner] / q_fd[inner] - 1)) < 1e-8
    # and the finite-difference Q approaches the analytic x0^2 + y0^2 + x0^-2
    q_exact = X ** 2 + Y ** 2 + X ** -2
    assert np.max(np.abs(o["Q"][inner] / q_exact[inner] - 1)) < 2 * d * d * 40


@pytest.mark.parametrize("way,tol", [(1, 5e-3), (2, 1e-8)])
def test_hyperbolic_method2(oracle_lib, way, tol):
    """Deviation vectors carry no finite-difference error: Q is the analytic
    value everywhere away from the top/side separatrix."""
    o, X, Y, d = _plane("hyperbolic", nu=64, method=2, way=way)
    top = np.abs(X) < 1 / math.e - 1e-3
    side = np.abs(X) > 1 / math.e + 1e-3
    assert np.max(np.abs(o["Q"][top] / E2 - 1)) < tol
    q_side = X ** 2 + Y ** 2 + X ** -2
    assert np.max(np.abs(o["Q"][side] / q_side[side] - 1)) < tol


@pytest.mark.parametrize("method,way,tol", [(1, 1, 1e-8), (2, 1, 1e-3), (2, 2, 1e-8)])
def test_expanding_field_pins_bn_ratio(oracle_lib, method, way, tol):
    """B=(x/2, 0, 1-z/2): Bz halves from bottom to top, so det D = 2 = |Bn1/Bn2|
    and Q = 2.5 for both top and side exits. A wrong normal-field factor in the
    Q assembly (Eq. Bn1) fails here."""
    o, X, Y, d = _plane("expanding", method=method, way=way)
    ok = np.abs(np.abs(X) - 0.5) > 2 * d
    assert np.all(o["status"][ok] == 0)
    assert np.max(np.abs(o["Q"][ok] / 2.5 - 1)) < tol
    top = np.abs(X) < 0.5 - 2 * d
    assert np.all(o["face2"][top] == 5)
    assert np.max(np.abs(o["r2"][top, 0] - 2 * X[top])) < 1e-8


@pytest.mark.parametrize("method,way,tol", [(1, 1, 1e-9), (2, 1, 1e-3), (2, 2, 1e-8)])
def test_shear_field_interior_plane(oracle_lib, method, way, tol):
    """B=(y/2, 0, 1) seeded on the interior plane z=1/2: x1 = x0 - y0/4,
    x2 = x0 + y0/4, so J1 is a non-symmetric shear and D = J2 J1^-1 has
    Q = 2 + 1/4. A transposed or misplaced adjugate (Eq. D+-3) fails here.
    Tw = -s/(4 pi sqrt(1 + s^2 y0^2)) with s = 1/2, length = sqrt(1 + y0^2/4)."""
    o, X, Y, d = _plane("shear", z=0.5, method=method, way=way)
    zz = np.abs(X) + 0.25 * np.abs(Y) < 1 - 2 * d
    assert np.all(o["face1"][zz] == 4) and np.all(o["face2"][zz] == 5)
    assert np.max(np.abs(o["Q"][zz] / 2.25 - 1)) < tol
    tw = -0.5 / (4 * math.pi * np.sqrt(1 + 0.25 * Y[zz] ** 2))
    assert np.max(np.abs(o["Tw"][zz] - tw)) < 1e-12
    assert np.max(np.abs(o["length"][zz] - np.sqrt(1 + 0.25 * Y[zz] ** 2))) < 1e-12
    assert np.max(np.abs(o["r1"][zz, 0] - (X[zz] - 0.25 * Y[zz]))) < 1e-10


def test_rigid_rotation_q_tw_length(oracle_lib):
    """B=(-qy, qx, 1), q=2 pi: lines with r0 < 1 make exactly one turn, so the
    footpoint is the seed lifted to z=1, Q = 2 and Tw = q/(2 pi sqrt(1+q^2 r0^2))
    (Tw = 1 on the axis), length = sqrt(1 + q^2 r0^2)."""
    o, X, Y, d = _plane("rotation", nu=64)
    R = np.hypot(X, Y)
    q = 2 * math.pi
    inn = R < 0.95
    assert np.all(o["status"][inn] == 0)
    assert np.max(np.abs(o["Q"][inn] - 2)) < 1e-8
    tw = q / (2 * math.pi * np.sqrt(1 + q * q * R ** 2))
    assert np.max(np.abs(o["Tw"][inn] - tw[inn])) < 1e-9
    assert np.max(np.abs(o["length"][inn] - np.sqrt(1 + q * q * R[inn] ** 2))) < 1e-9
    assert np.max(np.abs(o["r2"][inn, :2] - np.stack([X[inn], Y[inn]], 1))) < 1e-9


def test_rotation_axis_twist_is_one(oracle_lib):
    B = synth.analytic_cube("rotation")
    out = oracle.twist(B, G1, np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.5]]), oracle.params(tol=1e-10))
    assert np.allclose(out["Tw"], 1.0, rtol=0, atol=1e-9)
    assert np.allclose(out["length"], 1.0, atol=1e-9)


@pytest.mark.parametrize("method", [1, 2])
def test_tilted_field_rotated_s0(oracle_lib, method):
    """B=(1,0,0.02) on the interior plane z=1/2: |Bn0/B| = 0.02 < 0.05, so
    Method I rotates S0 perpendicular to B (Sec. 4) and traces 4 extra lines;
    straight parallel lines give Q = 2 exactly."""
    o, X, Y, d = _plane("tilted", z=0.5, method=method, way=2)
    if method == 1:
        assert np.all(o["status"] & oracle.ROTATED)
    assert np.max(np.abs(o["Q"] - 2)) < 1e-10
    assert np.all(o["face1"] == 0) and np.all(o["face2"] == 1)


def test_closed_loops_hit_max_steps(oracle_lib):
    B = synth.analytic_cube("loops")
    seeds = np.array([[0.5, 0.0, 0.5], [0.2, 0.1, 0.3]])
    out = oracle.twist(B, G1, seeds, oracle.params(tol=1e-6, max_steps=2000))
    assert np.all(out["status"] & oracle.MAXSTEPS)
    assert np.all(np.isnan(out["Tw"])) and np.all(out["steps"] == 2000)


def test_zero_field_and_outside_seeds(oracle_lib):
    B = synth.analytic_cube("zero")
    out = oracle.twist(B, G1, np.array([[0.0, 0.0, 0.5]]), oracle.params())
    assert out["status"][0] == oracle.NULL_B and np.isnan(out["Tw"][0])
    B = synth.analytic_cube("uniform")
    out = oracle.twist(B, G1, np.array([[0.0, 0.0, 1.5], [1.01, 0, 0.5]]), oracle.params())
    assert np.all(out["status"] == oracle.OUTSIDE)


def test_seed_on_face_has_zero_length_backward(oracle_lib):
    """Reading R6: a direction whose first step leaves through the seed's own
    face has length 0 and its footpoint is the seed."""
    B = synth.analytic_cube("hyperbolic")
    out = oracle.trace(B, G1, np.array([[0.1, 0.2, 0.0]]), 1e-10)
    e = out["ends"][0]
    assert out["faces"][0, 0] == 4
    assert np.all(e[0, :3] == np.array([(0.1 + 1) / G1.spacing[0], (0.2 + 1) / G1.spacing[1], 0.0]))
    assert e[0, 3] == 0.0 and e[0, 4] == 0.0


def test_exit_lands_exactly_on_face(oracle_lib):
    """Reading R5: the Henon step puts the footpoint's normal coordinate exactly
    on the face (index n-1, physical hi)."""
    rng = np.random.default_rng(7)
    B, grid = synth.random_smooth_cube(rng, n=(9, 9, 9))
    seeds = rng.uniform(0.1, 0.9, size=(50, 3))
    out = oracle.trace(B, grid, seeds, 1e-6)
    for s in range(50):
        for e in range(2):
            f = out["faces"][s, e]
            a = f // 2
            want = 0.0 if f % 2 == 0 else grid.n[a] - 1.0
            assert out["ends"][s, e, a] == want
            others = [b for b in range(3) if b != a]
            assert all(0 <= out["ends"][s, e, b] <= grid.n[b] - 1 for b in others)
