"""CUDA path vs the FP64 oracle on the same seeded inputs, through the C ABI.

FP64 tracer: every output (Q, Tw, length, footpoints, faces, status, step
counts) identical to the oracle's to the last bit, which implies the parity
bars (median relative Q/Tw error <= 1e-9, 99th percentile <= 1e-4 for
Q < 1e6, faces, status and footpoint cells exact); both are asserted. FP32
tracer: its error against the oracle is measured and bounded loosely (it is
reported, not gated at FP64 level)."""
import math

import numpy as np
import pytest

import oracle
import synth
from parity import (assert_bitwise, assert_exact_ints, assert_fp64_parity, footpoint_cells_exact, q_rel, to_np,
                    tw_rel)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_12569_gb300 as m

    return m


def _field(fq, B, grid):
    return fq.Field(torch.from_numpy(np.ascontiguousarray(B)).cuda(), grid.origin, grid.spacing)


def _gpu_plane(fq, field, origin, u, v, nu, nv, **kw):
    out = fq.qmap_plane(field, origin, u, v, nu, nv, fq.params(**kw))
    field.check()
    return to_np(out)


G1 = synth.ANALYTIC_GRID
D1 = 2.0 / 128


@pytest.mark.parametrize("kind", ["hyperbolic", "rotation", "uniform", "shear", "expanding"])
@pytest.mark.parametrize("tol", [1e-10, 10 ** -3.2])
def test_analytic_fp64_parity(fq, oracle_lib, kind, tol):
    """Analytic 64^3 fields, 128x128 cell-centred seeds on z=0."""
    B = synth.analytic_cube(kind)
    field = _field(fq, B, G1)
    args = ((-1.0, -1.0, 0.0), (D1, 0, 0), (0, D1, 0), 128, 128)
    g = _gpu_plane(fq, field, *args, precision="f64", tol=tol)
    r = oracle.plane(B, G1, *args, oracle.params(tol=tol))
    assert_fp64_parity(g, r)
    footpoint_cells_exact(g, r, G1)
    assert_bitwise(g, r)


def test_analytic_closed_forms_on_gpu(fq, oracle_lib):
    """The closed forms themselves, on the FP64 and FP32 paths."""
    X, Y = np.meshgrid(-1 + (np.arange(128) + 0.5) * D1, -1 + (np.arange(128) + 0.5) * D1, indexing="xy")
    X, Y = X.ravel(), Y.ravel()
    args = ((-1.0, -1.0, 0.0), (D1, 0, 0), (0, D1, 0), 128, 128)
    e2 = math.e ** 2 + math.e ** -2
    for prec, tolq in (("f64", 1e-8), ("f32", 2e-3)):
        field = _field(fq, synth.analytic_cube("hyperbolic"), G1)
        g = _gpu_plane(fq, field, *args, precision=prec, tol=1e-10 if prec == "f64" else 1e-5)
        top = np.abs(X) < 1 / math.e - 2 * D1
        assert np.max(np.abs(g["Q"][top] / e2 - 1)) < tolq
        field = _field(fq, synth.analytic_cube("rotation"), G1)
        g = _gpu_plane(fq, field, *args, precision=prec, tol=1e-10 if prec == "f64" else 1e-5)
        R = np.hypot(X, Y)
        inn = R < 0.95
        q = 2 * math.pi
        assert np.max(np.abs(g["Q"][inn] - 2)) < 2 * tolq
        assert np.max(np.abs(g["Tw"][inn] - q / (2 * math.pi * np.sqrt(1 + q * q * R[inn] ** 2)))) < tolq
        field = _field(fq, synth.analytic_cube("uniform"), G1)
        g = _gpu_plane(fq, field, *args, precision=prec)
        assert np.max(np.abs(g["Q"] - 2)) < 1e-6 and np.max(np.abs(g["Tw"])) < 1e-7


@pytest.fixture(scope="module")
def mono():
    grid = synth.Grid((64, 56, 32), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    ch = synth.random_charges(np.random.default_rng(2208), 10, ((0.0, 63.0), (0.0, 55.0)), depth=(4.0, 12.0))
    B = synth.monopole_cube(grid, ch, dtype=np.float32)
    return B, grid


def test_monopole_plane_fp64_parity_ragged(fq, oracle_lib, mono):
    """Several tiles and ragged tails (101 x 75 seeds, 8x4 tiles)."""
    B, grid = mono
    field = _field(fq, B, grid)
    nu, nv = 101, 75
    args = ((0.0, 0.0, 0.0), (63.0 / nu, 0, 0), (0, 55.0 / nv, 0), nu, nv)
    g = _gpu_plane(fq, field, *args, precision="f64")
    r = oracle.plane(B.astype(np.float64), grid, *args, oracle.params())
    assert_fp64_parity(g, r)
    footpoint_cells_exact(g, r, grid)
    assert_bitwise(g, r)


@pytest.mark.parametrize("precision", ["f32", "f32acc64"])
def test_monopole_plane_fp32_error_stated(fq, oracle_lib, mono, precision):
    B, grid = mono
    field = _field(fq, B, grid)
    nu, nv = 101, 75
    args = ((0.0, 0.0, 0.0), (63.0 / nu, 0, 0), (0, 55.0 / nv, 0), nu, nv)
    g = _gpu_plane(fq, field, *args, precision=precision)
    r = oracle.plane(B.astype(np.float64), grid, *args, oracle.params())
    assert np.mean(g["face2"] == r["face2"]) > 0.99
    rel = q_rel(g, r)
    both = np.isfinite(g["Q"]) & np.isfinite(r["Q"])
    assert np.mean(both) > 0.95
    assert np.median(rel[np.isfinite(rel)]) < 1e-3
    assert np.median(tw_rel(g, r)[np.isfinite(tw_rel(g, r))]) < 1e-4


def test_interior_plane_rotation_parity(fq, oracle_lib, mono):
    """A vertical interior plane (xz at y = 10.3): near-tangent seeds rotate S0
    and trace four extra lines (Sec. 4)."""
    B, grid = mono
    field = _field(fq, B, grid)
    nu, nv = 70, 36
    args = ((0.0, 10.3, 0.0), (63.0 / nu, 0, 0), (0, 0, 31.0 / nv), nu, nv)
    g = _gpu_plane(fq, field, *args, precision="f64")
    r = oracle.plane(B.astype(np.float64), grid, *args, oracle.params())
    assert (r["status"] & oracle.ROTATED).sum() > 50
    assert_fp64_parity(g, r)
    assert_bitwise(g, r)


def test_tilted_field_rotation_q2(fq, oracle_lib):
    B = synth.analytic_cube("tilted")
    field = _field(fq, B, G1)
    d = 2.0 / 32
    g = _gpu_plane(fq, field, (-1.0, -1.0, 0.5), (d, 0, 0), (0, d, 0), 32, 32, precision="f64", tol=1e-10)
    assert np.all(g["status"] & 32)
    assert np.max(np.abs(g["Q"] - 2)) < 1e-10


def test_volume_parity(fq, oracle_lib, mono):
    B, grid = mono
    field = _field(fq, B, grid)
    step = (63.0 / 20, 55.0 / 18, 31.0 / 6)
    g = to_np(fq.qmap_volume(field, (0.0, 0.0, 0.0), step, 20, 18, 6, fq.params(precision="f64")))
    field.check()
    r = oracle.qmap(B.astype(np.float64), grid, (0.0, 0.0, 0.0), (step[0], 0, 0), (0, step[1], 0), (0, 0, step[2]),
                    (20, 18, 6), oracle.params())
    assert (r["status"] & oracle.ROTATED).sum() > 0
    assert_fp64_parity(g, r)
    assert_bitwise(g, r)


def test_twist_list_parity(fq, oracle_lib, mono):
    B, grid = mono
    field = _field(fq, B, grid)
    rng = np.random.default_rng(3)
    seeds = np.concatenate([rng.uniform([0, 0, 0], [63, 55, 31], size=(500, 3)),
                            [[70.0, 1.0, 1.0], [-0.5, 3.0, 3.0]]])  # two outside the box
    g = to_np(fq.twist(field, torch.from_numpy(seeds).cuda(), fq.params(precision="f64")))
    field.check()
    r = oracle.twist(B.astype(np.float64), grid, seeds, oracle.params())
    assert_fp64_parity(g, r)
    assert_bitwise(g, r)
    assert np.all(g["status"][-2:] == 16)
    for k in ("r1", "r2"):
        ok = (r["status"] & 19) == 0
        assert np.max(np.abs(g[k][ok] - r[k][ok])) < 1e-6


def test_edge_cases(fq, oracle_lib):
    # closed loops stop at max_steps; zero field is NULL_B; single-seed lattice; empty list
    B = synth.analytic_cube("loops")
    field = _field(fq, B, G1)
    seeds = torch.tensor([[0.5, 0.0, 0.5]], dtype=torch.float64, device="cuda")
    for prec in ("f64", "f32"):
        g = to_np(fq.twist(field, seeds, fq.params(precision=prec, tol=1e-6, max_steps=2000)))
        assert g["status"][0] & 1 and np.isnan(g["Tw"][0]) and g["steps"][0] == 2000
    field = _field(fq, synth.analytic_cube("zero"), G1)
    g = _gpu_plane(fq, field, (-1.0, -1.0, 0.0), (D1, 0, 0), (0, D1, 0), 4, 4, precision="f64")
    assert np.all(g["status"] == 2) and np.all(np.isnan(g["Q"]))
    field = _field(fq, synth.analytic_cube("uniform"), G1)
    g = _gpu_plane(fq, field, (-0.5, -0.5, 0.0), (1.0, 0, 0), (0, 1.0, 0), 1, 1, precision="f64")
    assert g["status"][0] == 8 and np.isnan(g["Q"][0]) and abs(g["Tw"][0]) < 1e-12
    out = fq.twist(field, torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    assert out["Tw"].numel() == 0
    # a plane partly outside the box: the inside seed has no in-box neighbour
    # along u (MIXED), the others are OUTSIDE
    g = _gpu_plane(fq, field, (0.9, -0.1, 0.0), (0.1, 0, 0), (0, 0.1, 0), 4, 2, precision="f64")
    assert list(g["status"][:4]) == [8, 16, 16, 16]


def test_argument_errors(fq):
    field = _field(fq, synth.analytic_cube("uniform"), G1)
    with pytest.raises(fq.FqslError):
        fq.qmap_plane(field, (0, 0, 0), (1, 0, 0), (1, 0, 0), 2, 2)  # u parallel to v
    with pytest.raises(fq.FqslError):
        fq.qmap_plane(field, (0, 0, 0), (0.1, 0, 0), (0, 0.1, 0), 2, 2, fq.params(tol=-1.0))
    f32only = fq.Field(torch.from_numpy(synth.analytic_cube("uniform")).cuda(), G1.origin, G1.spacing,
                       pack=("f32",))
    with pytest.raises(fq.FqslError) as ei:
        fq.qmap_plane(f32only, (0, 0, 0), (0.1, 0, 0), (0, 0.1, 0), 2, 2, fq.params(precision="f64"))
    assert ei.value.status == 5
    # seed counts whose product overflows 64 bits (2^32 x 2^32 wraps to 0) are
    # refused before any launch
    small = fq.alloc_out(1)
    with pytest.raises(fq.FqslError) as ei:
        fq.qmap_plane(field, (0, 0, 0), (0.1, 0, 0), (0, 0.1, 0), 1 << 32, 1 << 32, out=small)
    assert ei.value.status == 1 and "2^31" in str(ei.value)
    with pytest.raises(fq.FqslError) as ei:
        fq.qmap_volume(field, (0, 0, 0), (0.1, 0.1, 0.1), 1 << 22, 1 << 21, 1 << 21, out=small)
    assert ei.value.status == 1 and "2^31" in str(ei.value)
    with pytest.raises(fq.FqslError) as ei:
        fq.Batch([field], [dict(origin=(0, 0, 0), u=(0.1, 0, 0), v=(0, 0.1, 0), nu=1 << 32, nv=1 << 32)],
                 outs=[small])
    assert ei.value.status == 1


def test_monopole_full_size_sampled_parity(fq, oracle_lib):
    """The benchmark workload at full size (256x256x128 FP32 monopole cube,
    1024x1024 seeds on z=0) in the benchmark's launch configuration; the oracle
    recomputes a seeded random sample of seeds one by one."""
    B, grid, _ = synth.monopole24_cube()
    field = _field(fq, B, grid)
    n = 1024
    args = ((0.0, 0.0, 0.0), (255.0 / n, 0, 0), (0, 255.0 / n, 0), n, n)
    g64 = _gpu_plane(fq, field, *args, precision="f64")
    g32 = _gpu_plane(fq, field, *args, precision="f32")
    sample = np.sort(np.random.default_rng(11).choice(n * n, 3000, replace=False))
    r = oracle.plane(B.astype(np.float64), grid, *args, oracle.params(), sample=sample)
    gs = {k: v[sample] for k, v in g64.items()}
    assert_fp64_parity(gs, r)
    assert_bitwise(gs, r)
    g32s = {k: v[sample] for k, v in g32.items()}
    assert np.mean(g32s["face2"] == r["face2"]) > 0.98
    rel = q_rel(g32s, r)
    assert np.median(rel[np.isfinite(rel)]) < 1e-3
    # the FP32 map's tail against the FP64 map at the same tolerance (3.2 % at
    # the 99th percentile over the whole map)
    assert np.percentile(rel[np.isfinite(rel)], 99) < 0.06


def test_monopole_fp32_accuracy_against_the_converged_map(fq, oracle_lib):
    """FP32 against the map itself: on the full-size benchmark map, both the
    FP32 and the FP64 map at the benchmark tolerance (10^-3.2) are compared
    with the oracle's map at tol_perp = 1e-10 on a seeded sample. FP64 at that
    tolerance carries the method's own integration error (a different step
    sequence than the converged one); FP32's error against the converged map
    must stay within twice FP64's, at the median and the 99th percentile, so
    that float rounding does not set the map's accuracy."""
    B, grid, _ = synth.monopole24_cube()
    field = _field(fq, B, grid)
    n = 1024
    args = ((0.0, 0.0, 0.0), (255.0 / n, 0, 0), (0, 255.0 / n, 0), n, n)
    g64 = _gpu_plane(fq, field, *args, precision="f64")
    g32 = _gpu_plane(fq, field, *args, precision="f32")
    sample = np.sort(np.random.default_rng(29).choice(n * n, 2000, replace=False))
    conv = oracle.plane(B.astype(np.float64), grid, *args, oracle.params(tol=1e-10), sample=sample)
    r32 = q_rel({k: v[sample] for k, v in g32.items()}, conv)
    r64 = q_rel({k: v[sample] for k, v in g64.items()}, conv)
    r32, r64 = r32[np.isfinite(r32)], r64[np.isfinite(r64)]
    assert len(r32) > 1900
    assert np.median(r64) > 1e-4  # the benchmark tolerance's own error is visible
    assert np.median(r32) <= 2.0 * np.median(r64)
    assert np.percentile(r32, 99) <= 2.0 * np.percentile(r64, 99)


# ---------------------------------------------------------------------------
# Method II (deviation vectors, Sec. 2.1 Eqs. rb2, q_scott; S0 perpendicular to
# B, Sec. 4), both ways of grad(B/|B|)
# ---------------------------------------------------------------------------
def _field_m2(fq, B, grid):
    return fq.Field(torch.from_numpy(np.ascontiguousarray(B)).cuda(), grid.origin, grid.spacing,
                    pack=("f32", "f64", "gradb"))


@pytest.mark.parametrize("way", [1, 2])
@pytest.mark.parametrize("kind,z", [("hyperbolic", 0.0), ("shear", 0.5), ("rotation", 0.0)])
def test_method2_analytic_fp64_bitwise(fq, oracle_lib, kind, z, way):
    B = synth.analytic_cube(kind)
    field = _field_m2(fq, B, G1)
    d = 2.0 / 64
    args = ((-1.0, -1.0, z), (d, 0, 0), (0, d, 0), 64, 64)
    g = _gpu_plane(fq, field, *args, precision="f64", method=2, gradb_way=way, tol=1e-9)
    r = oracle.plane(B, G1, *args, oracle.params(method=2, way=way, tol=1e-9))
    assert_fp64_parity(g, r)
    assert_bitwise(g, r)


@pytest.mark.parametrize("way", [1, 2])
def test_method2_monopole_fp64_bitwise_and_fp32(fq, oracle_lib, mono, way):
    B, grid = mono
    field = _field_m2(fq, B, grid)
    nu, nv = 61, 43
    args = ((0.0, 0.0, 0.0), (63.0 / nu, 0, 0), (0, 55.0 / nv, 0), nu, nv)
    g = _gpu_plane(fq, field, *args, precision="f64", method=2, gradb_way=way)
    r = oracle.plane(B.astype(np.float64), grid, *args, oracle.params(method=2, way=way))
    assert_fp64_parity(g, r)
    assert_bitwise(g, r)
    g32 = _gpu_plane(fq, field, *args, precision="f32", method=2, gradb_way=way)
    assert np.mean(g32["face2"] == r["face2"]) > 0.99
    rel = q_rel(g32, r)
    assert np.median(rel[np.isfinite(rel)]) < 1e-3


def test_method2_closed_form_on_gpu(fq, oracle_lib):
    """Deviation vectors carry no finite-difference error: on B=(x,-y,1) the
    top-exit Q is e^2 + e^-2 (way 2) on both precisions."""
    B = synth.analytic_cube("hyperbolic")
    field = _field_m2(fq, B, G1)
    X, Y = np.meshgrid(-1 + (np.arange(64) + 0.5) / 32, -1 + (np.arange(64) + 0.5) / 32, indexing="xy")
    X = X.ravel()
    top = np.abs(X) < 1 / math.e - 1e-3
    e2 = math.e ** 2 + math.e ** -2
    for prec, tol, bound in (("f64", 1e-10, 1e-8), ("f32", 1e-6, 2e-3)):
        g = _gpu_plane(fq, field, (-1.0, -1.0, 0.0), (1 / 32, 0, 0), (0, 1 / 32, 0), 64, 64, precision=prec,
                       method=2, gradb_way=2, tol=tol)
        assert np.max(np.abs(g["Q"][top] / e2 - 1)) < bound


def test_method2_volume_fp64_bitwise(fq, oracle_lib, mono):
    B, grid = mono
    field = _field_m2(fq, B, grid)
    step = (63.0 / 12, 55.0 / 10, 31.0 / 4)
    g = to_np(fq.qmap_volume(field, (0.0, 0.0, 0.0), step, 12, 10, 4, fq.params(precision="f64", method=2)))
    field.check()
    r = oracle.qmap(B.astype(np.float64), grid, (0.0, 0.0, 0.0), (step[0], 0, 0), (0, step[1], 0), (0, 0, step[2]),
                    (12, 10, 4), oracle.params(method=2))
    assert_bitwise(g, r)


@pytest.mark.parametrize("way,qperp", [(1, 0), (2, 0), (1, 1)], ids=["way1", "way2", "way1_qperp"])
def test_method2_monopole_full_size_sampled(fq, oracle_lib, way, qperp):
    """Method II (and Q_perp) on the benchmark's full-size map (256x256x128
    FP32 monopole cube, 1024x1024 seeds on z=0) in the launch the benchmark
    times: FP64 bit-identical to the oracle on a seeded sample of seeds, each
    recomputed on its own, and the FP32 error stated."""
    B, grid, _ = synth.monopole24_cube()
    field = _field_m2(fq, B, grid)
    n = 1024
    args = ((0.0, 0.0, 0.0), (255.0 / n, 0, 0), (0, 255.0 / n, 0), n, n)
    kw = dict(method=2, gradb_way=way, qperp=qperp)
    g64 = _gpu_plane(fq, field, *args, precision="f64", **kw)
    g32 = _gpu_plane(fq, field, *args, precision="f32", **kw)
    sample = np.sort(np.random.default_rng(13 + way + 2 * qperp).choice(n * n, 1500, replace=False))
    r = oracle.plane(B.astype(np.float64), grid, *args, oracle.params(method=2, way=way, qperp=qperp), sample=sample)
    gs = {k: v[sample] for k, v in g64.items()}
    assert_fp64_parity(gs, r)
    assert_bitwise(gs, r)
    g32s = {k: v[sample] for k, v in g32.items()}
    assert np.mean(g32s["face2"] == r["face2"]) > 0.98
    rel = q_rel(g32s, r)
    assert np.median(rel[np.isfinite(rel)]) < 1e-3


def test_method2_way1_needs_gradient_grid(fq):
    field = _field(fq, synth.analytic_cube("uniform"), G1)
    with pytest.raises(fq.FqslError) as ei:
        fq.qmap_plane(field, (-1, -1, 0), (0.1, 0, 0), (0, 0.1, 0), 4, 4, fq.params(method=2, gradb_way=1))
    assert ei.value.status == 5


# ---------------------------------------------------------------------------
# Q_perp: Method II with S1, S2 perpendicular to the line at its ends (Sec. 2.1
# after Titov 2007)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("way", [1, 2])
def test_qperp_monopole_fp64_bitwise_and_fp32(fq, oracle_lib, mono, way):
    B, grid = mono
    field = _field_m2(fq, B, grid)
    nu, nv = 61, 43
    args = ((0.0, 0.0, 0.0), (63.0 / nu, 0, 0), (0, 55.0 / nv, 0), nu, nv)
    g = _gpu_plane(fq, field, *args, precision="f64", method=2, gradb_way=way, qperp=1)
    r = oracle.plane(B.astype(np.float64), grid, *args, oracle.params(method=2, way=way, qperp=1))
    assert_fp64_parity(g, r)
    assert_bitwise(g, r)
    # Q_perp and the face Q are different numbers on this map
    rf = oracle.plane(B.astype(np.float64), grid, *args, oracle.params(method=2, way=way))
    ok = np.isfinite(r["Q"])
    assert np.median(np.abs(r["Q"][ok] / rf["Q"][ok] - 1)) > 1e-3
    g32 = _gpu_plane(fq, field, *args, precision="f32", method=2, gradb_way=way, qperp=1)
    rel = q_rel(g32, r)
    assert np.median(rel[np.isfinite(rel)]) < 1e-3


def test_qperp_interior_volume_fp64_bitwise(fq, oracle_lib, mono):
    B, grid = mono
    field = _field_m2(fq, B, grid)
    step = (63.0 / 12, 55.0 / 10, 31.0 / 4)
    g = to_np(fq.qmap_volume(field, (0.0, 0.0, 0.0), step, 12, 10, 4,
                             fq.params(precision="f64", method=2, qperp=1)))
    field.check()
    r = oracle.qmap(B.astype(np.float64), grid, (0.0, 0.0, 0.0), (step[0], 0, 0), (0, step[1], 0), (0, 0, step[2]),
                    (12, 10, 4), oracle.params(method=2, qperp=1))
    assert_bitwise(g, r)


def test_qperp_closed_form_on_gpu(fq, oracle_lib):
    # the rigid rotation maps perpendicular cross-sections isometrically:
    # Q_perp = 2. (FP32 way 2 differences B/|B| in float over 0.002 cells, and
    # the rounding of B/|B| it amplifies leaves about 1 % on these lines.)
    B = synth.analytic_cube("rotation")
    field = _field_m2(fq, B, G1)
    d = 0.5 / 16
    for prec, tol, bound in (("f64", 1e-10, 1e-6), ("f32", 1e-6, 2e-2)):
        g = _gpu_plane(fq, field, (-0.25, -0.25, 0.0), (d, 0, 0), (0, d, 0), 16, 16, precision=prec, method=2,
                       gradb_way=2, tol=tol, qperp=1)
        assert np.max(np.abs(g["Q"] / 2 - 1)) < bound


def test_qperp_needs_method2(fq):
    field = _field(fq, synth.analytic_cube("uniform"), G1)
    with pytest.raises(fq.FqslError) as ei:
        fq.qmap_plane(field, (-1, -1, 0), (0.1, 0, 0), (0, 0.1, 0), 4, 4, fq.params(qperp=1))
    assert ei.value.status == 5
