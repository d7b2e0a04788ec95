"""Pins of the oracle's Q_perp (reading R17: Method II with the end planes S1,
S2 perpendicular to the line, Sec. 2.1 after Titov 2007).

- closed forms: a uniform field and the rigid rotation (a screw motion maps
  perpendicular cross-sections isometrically) give Q_perp = 2; on the axis of
  the hyperbolic field B is normal to both end faces, so Q_perp = Q;
- brute force: Q_perp from central differences of four neighbouring lines
  traced at a tight tolerance, their end displacements projected onto the plane
  perpendicular to B at the centre line's ends, agrees with the deviation-vector
  value to O(delta^2) on a generic monopole field (and is >= 2 there).

On coarse maps both Method II forms can dip a little below 2 (to 1.96 on a
48x40x24 monopole map): trilinear interpolation of a solenoidal field is not
exactly solenoidal, so the flux through a thin tube, which the Bn
normalisation of Eq. q_scott assumes constant, drifts along the line.
"""
import math

import numpy as np

import oracle
import synth

G1 = synth.ANALYTIC_GRID
E2 = math.e ** 2 + math.e ** -2


def _m2(B, grid, plane, qperp, tol=1e-10, way=1):
    return oracle.plane(B, grid, *plane, oracle.params(method=2, way=way, tol=tol, qperp=qperp))


def test_uniform_and_rotation_give_two():
    # (the rotation field's B/|B| is far from linear on the 64^3 grid: the
    # gradient grid of way 1 is off by up to 10 % there, so way 2 carries the
    # closed form; way 1 is exact on the uniform field)
    d = 0.5 / 8
    plane = ((-0.25, -0.25, 0.0), (d, 0, 0), (0, d, 0), 8, 8)
    for kind, ways in (("uniform", (1, 2)), ("rotation", (2,))):
        B = synth.analytic_cube(kind)
        for way in ways:
            out = _m2(B, G1, plane, 1, way=way)
            assert np.all((out["status"] & oracle.BAD) == 0)
            np.testing.assert_allclose(out["Q"], 2.0, rtol=1e-6)


def test_hyperbolic_axis_equals_q():
    # lattice with a seed on the axis (x = y = 0): B = (0, 0, 1) there and at
    # both footpoints, so the perpendicular planes are the faces
    B = synth.analytic_cube("hyperbolic")
    # (way 2: B/|B| is not linear, so the gradient grid of way 1 is off by 2e-3)
    plane = ((-0.05, -0.05, 0.0), (0.1, 0, 0), (0, 0.1, 0), 1, 1)
    qp = _m2(B, G1, plane, 1, way=2)["Q"][0]
    q = _m2(B, G1, plane, 0, way=2)["Q"][0]
    np.testing.assert_allclose(qp, E2, rtol=1e-6)
    np.testing.assert_allclose(q, E2, rtol=1e-6)
    # off the axis the planes tilt and the two differ
    plane = ((0.35, 0.2, 0.0), (0.1, 0, 0), (0, 0.1, 0), 1, 1)
    assert abs(_m2(B, G1, plane, 1, way=2)["Q"][0] / _m2(B, G1, plane, 0, way=2)["Q"][0] - 1) > 1e-3


def _perp_frame(b):
    m = int(np.argmin(np.abs(b)))
    e = np.zeros(3)
    e[m] = 1.0
    u = np.cross(b, e)
    u /= np.linalg.norm(u)
    return u, np.cross(b, u)


def _basis(b):
    u, v = _perp_frame(b)
    return np.stack([u, v])


def test_brute_force_perpendicular_differences():
    grid = synth.Grid((40, 36, 24), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    rng = np.random.default_rng(9)
    ch = synth.random_charges(rng, 6, ((0.0, 39.0), (0.0, 35.0)), depth=(6.0, 12.0))
    B = synth.monopole_cube(grid, ch, dtype=np.float64)
    J = oracle.curl(B, grid)
    p = oracle.params(tol=1e-11, max_steps=10 ** 7)
    seeds = rng.uniform((8.0, 8.0, 6.0), (31.0, 27.0, 16.0), (12, 3))
    delta = 1e-3
    checked = 0
    rel = []
    for r0 in seeds:
        xi0 = (r0 - np.asarray(grid.origin)) / np.asarray(grid.spacing)
        B0 = oracle.interp(B, grid.n, xi0)[0]
        b0 = B0 / np.linalg.norm(B0)
        u, v = _perp_frame(b0)
        pts = np.stack([r0, r0 + delta * u, r0 - delta * u, r0 + delta * v, r0 - delta * v])
        tr = oracle.trace(B, grid, pts, 1e-11, p, J=J)
        if np.any(tr["status"] & oracle.BAD) or np.any(tr["faces"] != tr["faces"][0]):
            continue
        ends = np.asarray(grid.origin) + np.asarray(grid.spacing) * tr["ends"][:, :, :3]
        Jm = []
        nB = []
        for e in range(2):
            Be = tr["Bend"][0, e]
            be = Be / np.linalg.norm(Be)
            P = np.eye(3) - np.outer(be, be)
            E = _basis(be)
            cu = E @ (P @ (ends[1, e] - ends[2, e])) / (2 * delta)
            cv = E @ (P @ (ends[3, e] - ends[4, e])) / (2 * delta)
            Jm.append(np.stack([cu, cv], 1))
            nB.append(np.linalg.norm(Be))
        J1, J2 = Jm
        adj = np.array([[J1[1, 1], -J1[0, 1]], [-J1[1, 0], J1[0, 0]]])
        q_fd = np.sum((J2 @ adj) ** 2) * nB[0] * nB[1] / np.dot(B0, B0)
        # the deviation-vector value at the same seed (a one-seed lattice, S0 perpendicular to B)
        plane = (tuple(r0 - 0.5 * (u + v)), tuple(u), tuple(v), 1, 1)
        # (way 2: the derivative of the interpolated field, as the traced
        # neighbours see it; way 1's node-gradient grid differs from it by the
        # grid's own discretisation error)
        q_m2 = _m2(B, grid, plane, 1, tol=1e-11, way=2)["Q"][0]
        assert q_fd >= 2.0 - 1e-6
        rel.append(abs(q_m2 / q_fd - 1))
        # the face-based Q of the same line is a different number wherever the
        # ends are oblique
        checked += 1
    assert checked >= 8
    # O(delta^2) differences and way 2's own +-0.001-cell differences: 4e-6 to 1.6e-4
    assert max(rel) < 5e-4 and np.median(rel) < 5e-5
