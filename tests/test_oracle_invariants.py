"""Invariant pins of the oracle on a small synthetic potential field:
Q >= 2 (its theoretical minimum, Sec. 1), Q, Tw and length constant along a
line and equal at both footpoints (Eq. qline), Method I and Method II
agreeing on smooth regions (Sec. 2.1: Eq. q_scott is equivalent to Eq. Q+-),
and convergence as tol -> 0 (Sec. 2.3)."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def field():
    grid = synth.Grid((48, 48, 32), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    rng = np.random.default_rng(2208)
    ch = synth.random_charges(rng, 8, ((0.0, 47.0), (0.0, 47.0)), depth=(6.0, 16.0))
    B = synth.monopole_cube(grid, ch, dtype=np.float32).astype(np.float64)
    return B, grid, oracle.curl(B, grid)


def _bottom(B, grid, J, n, p, sample=None):
    d = 47.0 / n
    return oracle.plane(B, grid, (0.0, 0.0, 0.0), (d, 0, 0), (0, d, 0), n, n, p, sample=sample, J=J)


def test_q_at_least_two(oracle_lib, field):
    """Q = |D|^2/|det D| >= 2 for any map; with |det D| replaced by the normal
    field ratio (Eq. Bn1) it holds up to the flux-conservation error of the
    trilinear (not exactly solenoidal) interpolant."""
    B, grid, J = field
    o = _bottom(B, grid, J, 48, oracle.params(method=2, way=2, tol=1e-8))
    ok = np.isfinite(o["Q"])
    assert ok.mean() > 0.95
    assert np.min(o["Q"][ok]) > 1.95
    assert np.percentile(o["Q"][ok], 1) > 1.99


def _centre_q(B, grid, J, r, a1, a2, p, delta=0.01):
    """Method I Q at r from a 3x3 lattice of spacing delta centred on r."""
    a1 = np.asarray(a1, float) * delta
    a2 = np.asarray(a2, float) * delta
    origin = np.asarray(r, float) - 1.5 * a1 - 1.5 * a2
    return oracle.qmap(B, grid, origin, a1, a2, counts=(3, 3, 1), p=p, sample=[4], J=J)


def test_q_constant_along_line_exact_field(oracle_lib):
    """Eq. qline: Q is a property of the whole line. On a generic affine
    divergence-free field (reproduced exactly by trilinear interpolation, so flux
    is conserved and Eq. Bn1 is exact) Method I with a horizontal S0 through an
    interior point (Eq. D+-2 makes Q independent of S0) equals Method I on the
    bottom face at the line's footpoint and on the top face at the other one."""
    B = synth.analytic_cube("linear")
    grid = synth.ANALYTIC_GRID
    rng = np.random.default_rng(5)
    seeds = rng.uniform([-0.4, -0.4, 0.2], [0.4, 0.4, 0.8], size=(12, 3))
    p = oracle.params(method=1, tol=1e-12)
    good = 0
    for s in seeds:
        o = _centre_q(B, grid, None, s, (1, 0, 0), (0, 1, 0), p, delta=1e-3)
        assert o["status"][0] == 0 and o["face1"][0] == 4
        for r_end in (o["r1"][0], o["r2"][0]):
            e = _centre_q(B, grid, None, r_end, (1, 0, 0), (0, 1, 0), p, delta=1e-3)
            if e["status"][0] != 0 or o["face2"][0] != 5:
                continue
            assert abs(e["Q"][0] / o["Q"][0] - 1) < 1e-6
            assert abs(e["length"][0] / o["length"][0] - 1) < 1e-9
            good += 1
    assert good >= 8


def test_tw_length_constant_along_line_monopoles(oracle_lib, field):
    """Tw and length are line integrals (Eq. tw), so they agree between an
    interior seed and the line's footpoint to integration accuracy; Q agrees to
    the flux-conservation error of the trilinear interpolant (Eq. Bn1 assumes
    div B = 0, which the interpolant of sampled monopoles only approximates)."""
    B, grid, J = field
    rng = np.random.default_rng(5)
    seeds = rng.uniform([8, 8, 2], [40, 40, 10], size=(30, 3))
    p = oracle.params(method=1, tol=1e-12)
    good = 0
    for s in seeds:
        o = _centre_q(B, grid, J, s, (1, 0, 0), (0, 1, 0), p)
        if o["status"][0] != 0 or not (o["face1"][0] == 4 and o["Q"][0] < 100):
            continue
        e = _centre_q(B, grid, J, o["r1"][0], (1, 0, 0), (0, 1, 0), p)
        if e["status"][0] != 0:
            continue
        assert abs(e["Q"][0] / o["Q"][0] - 1) < 0.1
        assert abs(e["Tw"][0] - o["Tw"][0]) < 1e-9
        assert abs(e["length"][0] / o["length"][0] - 1) < 1e-9
        assert np.max(np.abs(e["r2"][0] - o["r2"][0])) < 1e-7
        good += 1
    assert good >= 10


def test_method2_q_constant_along_analytic_line(oracle_lib):
    """On B=(x,-y,1) (exactly trilinear) Method II from any interior point of a
    top-exiting line gives Q = e^2 + e^-2."""
    B = synth.analytic_cube("hyperbolic")
    p = oracle.params(method=2, way=2, tol=1e-11)
    e2 = np.e ** 2 + np.e ** -2
    for z0 in (0.0, 0.3, 0.7, 1.0):
        for x0, y0 in ((0.1, 0.2), (-0.2, -0.5)):
            r = np.array([x0 * np.exp(z0), y0 * np.exp(-z0), z0])
            lo = r - np.array([5e-4, 5e-4, 0.0])  # the single seed sits at lo + (a1 + a2)/2 = r
            o = oracle.qmap(B, synth.ANALYTIC_GRID, lo, (1e-3, 0, 0), (0, 1e-3, 0), counts=(1, 1, 1), p=p)
            assert abs(o["Q"][0] / e2 - 1) < 1e-8


def test_method1_method2_agree_on_smooth_regions(oracle_lib, field):
    """Sec. 2.1: Eq. q_scott is equivalent to Eq. Q+-. Method I (finite
    differences over a lattice step delta) converges to Method II as O(delta^2)."""
    B, grid, J = field
    pts = np.random.default_rng(1).uniform(4, 43, size=(60, 2))

    def m1(delta):
        return np.array([_centre_q(B, grid, J, (x, y, 0.0), (1, 0, 0), (0, 1, 0),
                                   oracle.params(method=1, tol=1e-11), delta=delta)["Q"][0] for x, y in pts])

    m2 = np.array([oracle.qmap(B, grid, (x - 5e-4, y - 5e-4, 0.0), (1e-3, 0, 0), (0, 1e-3, 0),
                               counts=(1, 1, 1), p=oracle.params(method=2, way=2, tol=1e-11), J=J)["Q"][0]
                   for x, y in pts])
    ok = np.isfinite(m2) & (m2 < 20)
    assert ok.sum() > 40
    err = {d: np.median(np.abs(m1(d)[ok] / m2[ok] - 1)) for d in (0.5, 0.25, 0.02)}
    assert err[0.02] < 1e-4
    assert err[0.5] / err[0.25] > 2.5  # second order in delta


def test_convergence_in_tol(oracle_lib, field):
    B, grid, J = field
    sample = np.arange(0, 48 * 48, 37)
    res = {t: _bottom(B, grid, J, 48, oracle.params(tol=t), sample=sample) for t in (1e-4, 1e-7, 1e-11)}
    ok = np.isfinite(res[1e-11]["Q"]) & np.isfinite(res[1e-4]["Q"]) & np.isfinite(res[1e-7]["Q"])
    e4 = np.median(np.abs(res[1e-4]["Q"][ok] / res[1e-11]["Q"][ok] - 1))
    e7 = np.median(np.abs(res[1e-7]["Q"][ok] / res[1e-11]["Q"][ok] - 1))
    assert e7 < e4 / 10
    assert np.median(res[1e-4]["steps"]) < np.median(res[1e-11]["steps"])


def test_sampled_equals_full_lattice(oracle_lib, field):
    B, grid, J = field
    p = oracle.params()
    full = _bottom(B, grid, J, 32, p)
    sample = np.array([0, 5, 31, 32, 500, 1023])
    part = _bottom(B, grid, J, 32, p, sample=sample)
    for k in ("Q", "Tw", "length", "r1", "r2", "face1", "face2", "status", "steps"):
        assert np.array_equal(full[k][sample], part[k], equal_nan=True), k
