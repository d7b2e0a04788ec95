"""The fixed-step scheme (Sec. 2.3: Kutta's 3/8-rule RK4; Sec. 4 Eq. step for
the per-line step; reading R18 of the oracle) on the CUDA path against the FP64
oracle, through the C ABI: FP64 bit-identical, FP32 error bounded."""
import math

import numpy as np
import pytest

import oracle
import synth
from parity import assert_bitwise, assert_fp64_parity, q_rel, to_np, tw_rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

G1 = synth.ANALYTIC_GRID
E2 = math.e ** 2 + math.e ** -2


@pytest.fixture(scope="module")
def fq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_12569_gb300 as m

    return m


@pytest.fixture(scope="module")
def mono():
    grid = synth.Grid((64, 56, 32), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    ch = synth.random_charges(np.random.default_rng(2208), 10, ((0.0, 63.0), (0.0, 55.0)), depth=(4.0, 12.0))
    return synth.monopole_cube(grid, ch, dtype=np.float32), grid


def _field(fq, B, grid, pack=("f32", "f64")):
    return fq.Field(torch.from_numpy(np.ascontiguousarray(B)).cuda(), grid.origin, grid.spacing, pack=pack)


def _plane(fq, field, *args, **kw):
    out = fq.qmap_plane(field, *args, fq.params(scheme=1, **kw))
    field.check()
    return to_np(out)


def _ora(**kw):
    return oracle.params(scheme=1, **kw)


@pytest.mark.parametrize("step", [3.0, 0.7])
def test_plane_fp64_bitwise_and_fp32(fq, oracle_lib, mono, step):
    B, grid = mono
    field = _field(fq, B, grid)
    nu, nv = 101, 75
    args = ((0.0, 0.0, 0.0), (63.0 / nu, 0, 0), (0, 55.0 / nv, 0), nu, nv)
    g = _plane(fq, field, *args, precision="f64", step=step)
    r = oracle.plane(B.astype(np.float64), grid, *args, _ora(step=step))
    assert_fp64_parity(g, r)
    assert_bitwise(g, r)
    for prec in ("f32", "f32acc64"):
        g32 = _plane(fq, field, *args, precision=prec, step=step)
        assert np.mean(g32["face2"] == r["face2"]) > 0.99
        rel = q_rel(g32, r)
        assert np.median(rel[np.isfinite(rel)]) < 1e-3
        t = tw_rel(g32, r)
        assert np.median(t[np.isfinite(t)]) < 1e-4


def test_interior_plane_rotation_fp64_bitwise(fq, oracle_lib, mono):
    B, grid = mono
    field = _field(fq, B, grid)
    args = ((0.0, 10.3, 0.0), (63.0 / 70, 0, 0), (0, 0, 31.0 / 36), 70, 36)
    g = _plane(fq, field, *args, precision="f64")
    r = oracle.plane(B.astype(np.float64), grid, *args, _ora())
    assert (r["status"] & oracle.ROTATED).sum() > 30
    assert_bitwise(g, r)


def test_volume_and_twist_fp64_bitwise(fq, oracle_lib, mono):
    B, grid = mono
    field = _field(fq, B, grid)
    step = (63.0 / 20, 55.0 / 18, 31.0 / 6)
    g = to_np(fq.qmap_volume(field, (0.0, 0.0, 0.0), step, 20, 18, 6, fq.params(precision="f64", scheme=1)))
    r = oracle.qmap(B.astype(np.float64), grid, (0.0, 0.0, 0.0), (step[0], 0, 0), (0, step[1], 0), (0, 0, step[2]),
                    (20, 18, 6), _ora())
    assert_bitwise(g, r)
    seeds = np.random.default_rng(3).uniform([0, 0, 0], [63, 55, 31], size=(300, 3))
    g = to_np(fq.twist(field, torch.from_numpy(seeds).cuda(), fq.params(precision="f64", scheme=1, step=1.3)))
    field.check()
    assert_bitwise(g, oracle.twist(B.astype(np.float64), grid, seeds, _ora(step=1.3)))


@pytest.mark.parametrize("way", [1, 2])
def test_method2_fp64_bitwise(fq, oracle_lib, mono, way):
    # Method II with step = 4.0 (the paper's Table 1 setting for way 1)
    B, grid = mono
    field = fq.Field(torch.from_numpy(B).cuda(), grid.origin, grid.spacing, pack=("f32", "f64", "gradb"))
    args = ((0.0, 0.0, 0.0), (63.0 / 61, 0, 0), (0, 55.0 / 43, 0), 61, 43)
    g = _plane(fq, field, *args, precision="f64", method=2, gradb_way=way, step=4.0)
    r = oracle.plane(B.astype(np.float64), grid, *args, _ora(method=2, way=way, step=4.0))
    assert_bitwise(g, r)


def test_closed_form_on_gpu(fq, oracle_lib):
    B = synth.analytic_cube("hyperbolic")
    field = _field(fq, B, G1)
    d = 0.6 / 24
    args = ((-0.3, -0.3, 0.0), (d, 0, 0), (0, d, 0), 24, 24)
    for prec, bound in (("f64", 1e-6), ("f32", 2e-3)):
        g = _plane(fq, field, *args, precision=prec, step=0.2, step_min=0.01)
        assert np.all(g["face2"] == 5)
        np.testing.assert_allclose(g["Q"], E2, rtol=bound)


def test_monopole_full_size_sampled(fq, oracle_lib):
    """The fixed-step map the benchmark times (the 256x256x128 FP32 monopole
    cube, 1024x1024 seeds on z=0, step_perp = 3 cells scaled by Eq. step) at
    full size: FP64 bit-identical to the oracle on a seeded sample of seeds,
    FP32 error stated."""
    B, grid, _ = synth.monopole24_cube()
    field = _field(fq, B, grid)
    n = 1024
    args = ((0.0, 0.0, 0.0), (255.0 / n, 0, 0), (0, 255.0 / n, 0), n, n)
    g64 = _plane(fq, field, *args, precision="f64", step=3.0)
    g32 = _plane(fq, field, *args, precision="f32", step=3.0)
    sample = np.sort(np.random.default_rng(12).choice(n * n, 3000, replace=False))
    r = oracle.plane(B.astype(np.float64), grid, *args, _ora(step=3.0), sample=sample)
    gs = {k: v[sample] for k, v in g64.items()}
    assert_fp64_parity(gs, r)
    assert_bitwise(gs, r)
    g32s = {k: v[sample] for k, v in g32.items()}
    assert np.mean(g32s["face2"] == r["face2"]) > 0.98
    rel = q_rel(g32s, r)
    assert np.median(rel[np.isfinite(rel)]) < 1e-3


def test_argument_errors(fq, mono):
    B, grid = mono
    field = _field(fq, B, grid)
    args = ((0.0, 0.0, 0.0), (1.0, 0, 0), (0, 1.0, 0), 4, 4)
    for kw, status in ((dict(scheme=2), 1), (dict(scheme=1, step=0.0), 1), (dict(scheme=1, step_min=5.0), 1)):
        with pytest.raises(fq.FqslError) as ei:
            fq.qmap_plane(field, *args, fq.params(**kw))
        assert ei.value.status == status, kw


def test_edge_cases_bitwise(fq, oracle_lib):
    # closed loops hit max_steps, a zero field is NULL_B, a plane partly
    # outside the box gives OUTSIDE and MIXED, the tilted field rotates S0
    cases = [
        ("loops", ((-0.5, -0.5, 0.5), (0.25, 0, 0), (0, 0.25, 0), 4, 4), dict(max_steps=3000, step=0.5)),
        ("zero", ((-0.5, -0.5, 0.0), (0.25, 0, 0), (0, 0.25, 0), 4, 4), {}),
        ("uniform", ((0.8, -0.2, 0.0), (0.2, 0, 0), (0, 0.2, 0), 4, 2), {}),
        ("tilted", ((-0.8, -0.8, 0.5), (0.1, 0, 0), (0, 0.1, 0), 16, 16), dict(step=0.3)),
    ]
    for kind, plane, kw in cases:
        B = synth.analytic_cube(kind)
        field = _field(fq, B, G1)
        gg = _plane(fq, field, *plane, precision="f64", **kw)
        r = oracle.plane(B, G1, *plane, _ora(**kw))
        assert_bitwise(gg, r)
        if kind == "loops":
            assert np.all(gg["status"] & oracle.MAXSTEPS)
        if kind == "zero":
            assert np.all(gg["status"] == oracle.NULL_B)
        if kind == "uniform":
            assert (gg["status"] & oracle.OUTSIDE).any() and (gg["status"] & oracle.MIXED).any()
        if kind == "tilted":
            assert np.all(gg["status"] & oracle.ROTATED)
            np.testing.assert_allclose(gg["Q"], 2.0, rtol=1e-6)
        field.close()
