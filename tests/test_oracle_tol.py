"""Pins of the per-line tolerance of Method I (Sec. 4, Eq. tol; reading R9):

    tol_line = tol_perp * max(|Bn0/B|, rot_thresh) ** tol_exp

on a box-face S0, and tol_line = tol_perp with S0 rotated perpendicular to B
where an interior S0 has |Bn0/B| < rot_thresh.

Every expected value here comes from the closed form of the field at the seed,
never from the oracle: the fields are linear (trilinear interpolation
reproduces them), so |Bn0/B| at a seed is known analytically. The oracle's
per-seed tolerance is read from its lattice step log. A plausible slip in the
oracle's formula -- an exponent of 1 or 2 instead of 1.5, an inverted ratio,
a dropped floor, the floor applied on an interior plane, or the ratio taken
against n0 of the wrong sign -- fails one of these tests. The last test checks
that the lattice lines are traced with that tolerance: their footpoints equal
those of a raw trace given the closed-form tolerance, and differ from traces
given the tolerances of the plausible slips.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import adjoint as oadj

TOL_PERP = 10 ** -3.2
GRID = synth.Grid((17, 17, 17), (-1.0, -1.0, 0.0), (0.125, 0.125, 1.0 / 16))


def _linear_cube(grid, fn):
    """Sample B = fn(X, Y, Z) (a linear field) at the grid's nodes."""
    x, y, z = (grid.axis(a) for a in range(3))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.ascontiguousarray(np.stack(fn(X, Y, Z), axis=-1).astype(np.float64))


def _log_tol(B, grid, origin, u, v, nu, nv, **kw):
    p = oracle.params(**{"tol": TOL_PERP, **kw})
    lg = oadj.lattice_log(B, grid, origin, u, v, nu, nv, p, cap=4096, extra=False)
    return lg["tol"], lg["status"]


def _seeds(origin, u, v, nu, nv):
    i, j = np.meshgrid(np.arange(nu), np.arange(nv), indexing="xy")
    i, j = i.ravel(), j.ravel()
    o, u, v = (np.asarray(a, float) for a in (origin, u, v))
    return o + (i[:, None] + 0.5) * u + (j[:, None] + 0.5) * v


@pytest.mark.parametrize("a", [0.0, 0.5, 1.0, 3.0, 10.0, 19.0, 30.0, 200.0])
def test_uniform_tilted_field_on_the_bottom_face(oracle_lib, a):
    """B = (a, 0, 1), S0 = the z = 0 face: |Bn0/B| = (1 + a^2)^(-1/2). Below
    the 0.05 floor (a = 30, 200) the floor applies and S0 is not rotated (a face
    plane)."""
    B = _linear_cube(GRID, lambda X, Y, Z: (a + 0 * X, 0 * X, 1 + 0 * X))
    tol, st = _log_tol(B, GRID, (-1.0, -1.0, 0.0), (0.25, 0, 0), (0, 0.25, 0), 8, 8)
    ratio = (1.0 + a * a) ** -0.5
    expect = TOL_PERP * max(ratio, 0.05) ** 1.5
    assert np.all(st & oracle.ROTATED == 0)
    assert np.allclose(tol, expect, rtol=1e-13, atol=0)
    if a >= 30.0:
        assert np.allclose(tol, TOL_PERP * 0.05 ** 1.5, rtol=1e-13)


@pytest.mark.parametrize("tol_exp", [1.0, 2.0, 0.5])
@pytest.mark.parametrize("rot_thresh", [0.05, 0.2])
def test_exponent_and_floor_parameters(oracle_lib, tol_exp, rot_thresh):
    """The same on B = (a, b, 1) over several tilts, with the exponent and the
    floor as parameters of Eq. tol."""
    for a, b in [(0.3, 0.1), (2.0, -1.0), (8.0, 6.0), (40.0, 1.0)]:
        B = _linear_cube(GRID, lambda X, Y, Z: (a + 0 * X, b + 0 * X, 1 + 0 * X))
        tol, _ = _log_tol(B, GRID, (-1.0, -1.0, 0.0), (0.5, 0, 0), (0, 0.5, 0), 4, 4, tol_exp=tol_exp,
                          rot_thresh=rot_thresh)
        ratio = (1.0 + a * a + b * b) ** -0.5
        assert np.allclose(tol, TOL_PERP * max(ratio, rot_thresh) ** tol_exp, rtol=1e-13, atol=0)


def test_varying_obliquity_across_a_face_plane(oracle_lib):
    """B = (s x, -s y, 1) with s = 40 on the z = 0 face: |Bn0/B| =
    1/sqrt(1 + s^2 (x^2 + y^2)) runs from 1/3 next to the centre to below the
    floor over most of the plane, seed by seed."""
    s = 40.0
    B = _linear_cube(GRID, lambda X, Y, Z: (s * X, -s * Y, 1 + 0 * X))
    org, u, v, nu, nv = (-1.0, -1.0, 0.0), (2.0 / 20, 0, 0), (0, 2.0 / 20, 0), 20, 20
    tol, st = _log_tol(B, GRID, org, u, v, nu, nv)
    r = _seeds(org, u, v, nu, nv)
    ratio = 1.0 / np.sqrt(1.0 + s * s * (r[:, 0] ** 2 + r[:, 1] ** 2))
    floor = ratio < 0.05
    assert floor.sum() > 100 and (~floor).sum() > 50 and ratio.max() > 0.3
    assert np.all(st & oracle.ROTATED == 0)
    assert np.allclose(tol, TOL_PERP * np.maximum(ratio, 0.05) ** 1.5, rtol=1e-12, atol=0)


def test_interior_tilted_plane_rotates_below_the_threshold(oracle_lib):
    """An interior S0 tilted by theta about y (n0 = (-sin, 0, cos)) in B =
    (s x, -s y, 1): |Bn0/B| = |cos - s x sin| / |B|. Seeds above the threshold
    take tol_perp |Bn0/B|^1.5 (no floor involved), seeds below rotate S0 and
    take tol_perp itself."""
    s, th = 3.0, 0.6
    B = _linear_cube(GRID, lambda X, Y, Z: (s * X, -s * Y, 1 + 0 * X))
    c, sn = math.cos(th), math.sin(th)
    d = 0.08
    org, u, v, nu, nv = (-0.2, -0.7, 0.15), (d * c, 0, d * sn), (0, d, 0), 15, 17
    tol, st = _log_tol(B, GRID, org, u, v, nu, nv)
    r = _seeds(org, u, v, nu, nv)
    assert np.all((r[:, 2] > 0.05) & (r[:, 2] < 0.95))
    Bs = np.stack([s * r[:, 0], -s * r[:, 1], np.ones(len(r))], 1)
    n0 = np.array([-sn, 0.0, c])
    ratio = np.abs(Bs @ n0) / np.linalg.norm(Bs, axis=1)
    rot = ratio < 0.05
    ok = st & oracle.BAD == 0
    assert rot.sum() >= 5 and (~rot).sum() > 100
    assert np.array_equal((st & oracle.ROTATED != 0)[ok], rot[ok])
    assert np.allclose(tol[~rot], TOL_PERP * ratio[~rot] ** 1.5, rtol=1e-12, atol=0)
    assert np.all(tol[rot] == TOL_PERP)


def test_lattice_lines_take_the_closed_form_tolerance(oracle_lib):
    """The tolerance is the one the lattice lines are traced with: on the z = 0
    face of B = (s x, -s y, 1), each line's top footpoint equals that of a
    raw trace from its seed given the closed-form tol_line (up to the one-ulp
    differences of tol that the ratio's rounding can make), and is farther
    from the traces given the tolerances of an exponent of 1 or 2 or of a
    dropped floor."""
    s = 6.0
    B = _linear_cube(GRID, lambda X, Y, Z: (s * X, -s * Y, 1 + 0 * X))
    org, u, v, nu, nv = (-0.6, -0.6, 0.0), (1.2 / 12, 0, 0), (0, 1.2 / 12, 0), 12, 12
    p = oracle.params(tol=1e-3)
    out = oracle.plane(B, GRID, org, u, v, nu, nv, p)
    r = _seeds(org, u, v, nu, nv)
    ratio = 1.0 / np.sqrt(1.0 + s * s * (r[:, 0] ** 2 + r[:, 1] ** 2))
    assert ratio.min() < 0.3

    def top(tol):
        t = oracle.trace(B, GRID, r, tol, oracle.params(tol=1e-3))
        return oracle.physical(GRID, t["ends"][:, 1, :3])

    ok = out["status"] & oracle.BAD == 0
    d_cf = np.abs(out["r2"] - top(1e-3 * np.maximum(ratio, 0.05) ** 1.5)).max(1)[ok]
    assert np.median(d_cf) < 1e-12 and d_cf.max() < 1e-6
    for wrong in (1e-3 * ratio ** 1.0, 1e-3 * ratio ** 2.0, 1e-3 * np.full_like(ratio, 1.0)):
        d_w = np.abs(out["r2"] - top(wrong)).max(1)[ok]
        assert np.median(d_w) > 1e3 * max(np.median(d_cf), 1e-12)


def test_floor_drop_is_seen_by_the_trace(oracle_lib):
    """Below the floor on a face plane: B = (-q y, q x, 1) with q = 40 makes
    helices that climb slowly (6.4 turns over the box height), and the seeds at
    r = 0.55 .. 0.9 have |Bn0/B| = 1/sqrt(1 + q^2 r^2) = 0.045 .. 0.028. Their
    footpoints are those of tol_perp 0.05^1.5 and not of tol_perp |Bn0/B|^1.5
    (the floor dropped)."""
    q = 40.0
    B = _linear_cube(GRID, lambda X, Y, Z: (-q * Y, q * X, 1 + 0 * X))
    org, u, v, nu, nv = (0.55, -0.15, 0.0), (0.05, 0, 0), (0, 0.05, 0), 7, 6
    p = oracle.params(tol=1e-2)
    out = oracle.plane(B, GRID, org, u, v, nu, nv, p)
    r = _seeds(org, u, v, nu, nv)
    ratio = 1.0 / np.sqrt(1.0 + q * q * (r[:, 0] ** 2 + r[:, 1] ** 2))
    assert ratio.max() < 0.05
    ok = out["status"] & oracle.BAD == 0
    assert ok.sum() > 30

    def far_end(tol):
        t = oracle.trace(B, GRID, r, tol, oracle.params(tol=1e-2))
        return oracle.physical(GRID, t["ends"][:, 1, :3])

    d_floor = np.abs(out["r2"] - far_end(np.full(len(r), 1e-2 * 0.05 ** 1.5))).max(1)[ok]
    d_drop = np.abs(out["r2"] - far_end(1e-2 * ratio ** 1.5)).max(1)[ok]
    assert d_floor.max() < 1e-9  # the seeds' own rounding, not the step sequence
    assert np.median(d_drop) > 1e-7
