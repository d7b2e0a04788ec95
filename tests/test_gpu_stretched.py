"""Stretched (rectilinear) grids on the CUDA path against the FP64 oracle on the
same seeded inputs, through the C ABI (fqsl_field_create_rect; Sec. 2.2 cell
search and Eqs. interp, w0, w1; Sec. 2.3 per-cell step and tolerance scaling;
reading R16 of the oracle).

FP64 tracer: every output identical to the oracle's to the last bit (so the
parity bars hold too; both are asserted). FP32 tracer: its error against the
oracle is bounded as on uniform grids. Method I, seed lists and Method II
(both ways of grad(B/|B|), Q and Q_perp)."""
import math

import numpy as np
import pytest

import oracle
import synth
from parity import assert_bitwise, assert_fp64_parity, q_rel, to_np, tw_rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E2 = math.e ** 2 + math.e ** -2


@pytest.fixture(scope="module")
def fq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_12569_gb300 as m

    return m


def _field(fq, B, grid, **kw):
    return fq.Field(torch.from_numpy(np.ascontiguousarray(B)).cuda(), coords=grid.coords, **kw)


def _plane(fq, field, *args, **kw):
    out = fq.qmap_plane(field, *args, fq.params(**kw))
    field.check()
    return to_np(out)


@pytest.fixture(scope="module")
def mono():
    # 64 x 56 x 32 nodes over [0, 63] x [0, 55] x [0, 31]: horizontal cells
    # growing 3 % per cell from the middle, vertical 4 % per cell upward
    grid = synth.stretched_grid((64, 56, 32), (0.0, 0.0, 0.0), (63.0, 55.0, 31.0), ratios=(1.03, 1.03, 1.04))
    ch = synth.random_charges(np.random.default_rng(2208), 10, ((0.0, 63.0), (0.0, 55.0)), depth=(4.0, 12.0))
    B = synth.monopole_cube(grid, ch, dtype=np.float32)
    return B, grid


def _cells_exact(g, r, grid, margin=1e-9):
    # footpoint cells (cell search of the oracle) agree except within margin
    # (relative to the cell width) of a node
    ok = (r["status"] & 19) == 0
    for k in ("r1", "r2"):
        for a in range(3):
            X = grid.axis(a)
            cr = oracle.cell_rect(X, r[k][ok, a])
            cg = oracle.cell_rect(X, g[k][ok, a])
            w = X[cr + 1] - X[cr]
            near = np.minimum(np.abs(r[k][ok, a] - X[cr]), np.abs(X[cr + 1] - r[k][ok, a])) < margin * w
            assert np.all((cr == cg) | near)


def test_plane_fp64_bitwise_ragged(fq, oracle_lib, mono):
    """z = 0 plane, several 8x4 tiles and ragged tails (101 x 75 seeds)."""
    B, grid = mono
    field = _field(fq, B, grid)
    nu, nv = 101, 75
    args = ((0.0, 0.0, 0.0), (63.0 / nu, 0, 0), (0, 55.0 / nv, 0), nu, nv)
    g = _plane(fq, field, *args, precision="f64")
    r = oracle.plane(B.astype(np.float64), grid, *args, oracle.params())
    assert np.isfinite(r["Q"]).sum() > 6000
    assert_fp64_parity(g, r)
    _cells_exact(g, r, grid)
    assert_bitwise(g, r)


@pytest.mark.parametrize("precision", ["f32", "f32acc64"])
def test_plane_fp32_error_stated(fq, oracle_lib, mono, precision):
    B, grid = mono
    field = _field(fq, B, grid)
    nu, nv = 101, 75
    args = ((0.0, 0.0, 0.0), (63.0 / nu, 0, 0), (0, 55.0 / nv, 0), nu, nv)
    g = _plane(fq, field, *args, precision=precision)
    r = oracle.plane(B.astype(np.float64), grid, *args, oracle.params())
    assert np.array_equal(g["status"] & oracle.BAD, r["status"] & oracle.BAD)
    assert np.mean(g["face2"] == r["face2"]) > 0.99
    rel = q_rel(g, r)
    assert np.mean(np.isfinite(g["Q"]) & np.isfinite(r["Q"])) > 0.95
    assert np.median(rel[np.isfinite(rel)]) < 1e-3
    t = tw_rel(g, r)
    assert np.median(t[np.isfinite(t)]) < 1e-4


def test_interior_plane_rotation_fp64_bitwise(fq, oracle_lib, mono):
    """A vertical interior plane: near-tangent seeds rotate S0 and trace four
    extra lines (Sec. 4) on the stretched grid."""
    B, grid = mono
    field = _field(fq, B, grid)
    nu, nv = 70, 36
    args = ((0.0, 10.3, 0.0), (63.0 / nu, 0, 0), (0, 0, 31.0 / nv), nu, nv)
    g = _plane(fq, field, *args, precision="f64")
    r = oracle.plane(B.astype(np.float64), grid, *args, oracle.params())
    assert (r["status"] & oracle.ROTATED).sum() > 30
    assert_fp64_parity(g, r)
    assert_bitwise(g, r)


def test_volume_fp64_bitwise(fq, oracle_lib, mono):
    B, grid = mono
    field = _field(fq, B, grid)
    step = (63.0 / 20, 55.0 / 18, 31.0 / 6)
    g = to_np(fq.qmap_volume(field, (0.0, 0.0, 0.0), step, 20, 18, 6, fq.params(precision="f64")))
    field.check()
    r = oracle.qmap(B.astype(np.float64), grid, (0.0, 0.0, 0.0), (step[0], 0, 0), (0, step[1], 0), (0, 0, step[2]),
                    (20, 18, 6), oracle.params())
    assert_bitwise(g, r)


def test_twist_list_fp64_bitwise(fq, oracle_lib, mono):
    B, grid = mono
    field = _field(fq, B, grid)
    rng = np.random.default_rng(3)
    seeds = np.concatenate([rng.uniform([0, 0, 0], [63, 55, 31], size=(500, 3)),
                            [[70.0, 1.0, 1.0], [-0.5, 3.0, 3.0], [0.0, 0.0, 0.0], [63.0, 55.0, 31.0]]])
    g = to_np(fq.twist(field, torch.from_numpy(seeds).cuda(), fq.params(precision="f64")))
    field.check()
    r = oracle.twist(B.astype(np.float64), grid, seeds, oracle.params())
    assert_bitwise(g, r)
    assert np.all(g["status"][-4:-2] == 16)


def test_closed_forms_on_gpu(fq, oracle_lib):
    # linear fields are exact under trilinear interpolation on any grid
    grid = synth.stretched_grid((40, 36, 30), (-1.0, -1.0, 0.0), (1.0, 1.0, 1.0), ratios=(1.04, 1.05, 1.06))
    d = 0.6 / 24
    xs = -0.3 + (np.arange(24) + 0.5) * d
    X, Y = (v.ravel() for v in np.meshgrid(xs, xs, indexing="xy"))
    field = _field(fq, synth.analytic_cube("hyperbolic", grid), grid)
    args = ((-0.3, -0.3, 0.0), (d, 0, 0), (0, d, 0), 24, 24)
    for prec, tol, qtol in (("f64", 1e-10, 1e-8), ("f32", 10 ** -3.2, 2e-3)):
        g = _plane(fq, field, *args, precision=prec, tol=tol)
        assert np.all((g["status"] & oracle.BAD) == 0) and np.all(g["face2"] == 5)
        np.testing.assert_allclose(g["Q"], E2, rtol=qtol)
    g = _plane(fq, field, *args, precision="f64", tol=1e-10)
    np.testing.assert_allclose(g["r2"][:, 0], X * math.e, rtol=0, atol=1e-8)
    np.testing.assert_allclose(g["r2"][:, 1], Y / math.e, rtol=0, atol=1e-8)
    q = 2.0 * math.pi
    field = _field(fq, synth.analytic_cube("rotation", grid, q=q), grid)
    g = _plane(fq, field, *args, precision="f64", tol=1e-10)
    r2 = X * X + Y * Y
    np.testing.assert_allclose(g["Tw"], q / (2 * math.pi * np.sqrt(1 + q * q * r2)), rtol=1e-7)


def test_uniform_coordinates_match_the_uniform_field(fq, oracle_lib, mono):
    # a stretched handle with uniform coordinates agrees with the uniform
    # handle of the same cube to the integration error (different rounding of
    # the same method); the FP64 stretched map is still the oracle's bit for bit
    B, _ = mono
    ug = synth.Grid((64, 56, 32), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    rg = synth.RectGrid(tuple(tuple(float(v) for v in ug.axis(a)) for a in range(3)))
    args = ((0.0, 0.0, 0.0), (63.0 / 48, 0, 0), (0, 55.0 / 40, 0), 48, 40)
    fu = fq.Field(torch.from_numpy(B).cuda(), ug.origin, ug.spacing)
    fr = _field(fq, B, rg)
    a = _plane(fq, fu, *args, precision="f64", tol=1e-10)
    b = _plane(fq, fr, *args, precision="f64", tol=1e-10)
    assert np.array_equal(a["face2"], b["face2"])
    ok = np.isfinite(a["Q"]) & np.isfinite(b["Q"])
    assert np.median(np.abs(b["Q"][ok] / a["Q"][ok] - 1)) < 1e-7
    assert_bitwise(b, oracle.plane(B.astype(np.float64), rg, *args, oracle.params(tol=1e-10)))


def test_static_entry_point(fq, oracle_lib, mono):
    # the allocation-free entry point serves stretched handles too
    B, grid = mono
    field = _field(fq, B, grid)
    args = ((0.0, 0.0, 0.0), (63.0 / 40, 0, 0), (0, 55.0 / 30, 0), 40, 30)
    out = fq.alloc_out(40 * 30)
    fq.qmap_plane_static(field, *args, fq.params(precision="f64"), out=out)
    field.check()
    assert_bitwise(to_np(out), oracle.plane(B.astype(np.float64), grid, *args, oracle.params()))


@pytest.mark.parametrize("way", [1, 2])
@pytest.mark.parametrize("qperp", [0, 1])
def test_method2_fp64_bitwise_and_fp32(fq, oracle_lib, mono, way, qperp):
    """Method II (deviation vectors) on the stretched grid: the gradient grid
    of way 1 with non-uniform stencils, way 2's offsets in cells of the step's
    start cell; Q and Q_perp."""
    B, grid = mono
    field = _field(fq, B, grid, pack=("f32", "f64", "gradb"))
    args = ((0.0, 0.0, 0.0), (63.0 / 61, 0, 0), (0, 55.0 / 43, 0), 61, 43)
    g = _plane(fq, field, *args, precision="f64", method=2, gradb_way=way, qperp=qperp)
    r = oracle.plane(B.astype(np.float64), grid, *args, oracle.params(method=2, way=way, qperp=qperp))
    assert np.isfinite(r["Q"]).sum() > 2000
    assert_fp64_parity(g, r)
    assert_bitwise(g, r)
    g32 = _plane(fq, field, *args, precision="f32", method=2, gradb_way=way, qperp=qperp)
    assert np.mean(g32["face2"] == r["face2"]) > 0.99
    rel = q_rel(g32, r)
    assert np.median(rel[np.isfinite(rel)]) < 1e-3


def test_method2_volume_fp64_bitwise(fq, oracle_lib, mono):
    B, grid = mono
    field = _field(fq, B, grid, pack=("f64", "gradb"))
    step = (63.0 / 12, 55.0 / 10, 31.0 / 4)
    g = to_np(fq.qmap_volume(field, (0.0, 0.0, 0.0), step, 12, 10, 4, fq.params(precision="f64", method=2)))
    field.check()
    r = oracle.qmap(B.astype(np.float64), grid, (0.0, 0.0, 0.0), (step[0], 0, 0), (0, step[1], 0), (0, 0, step[2]),
                    (12, 10, 4), oracle.params(method=2))
    assert_bitwise(g, r)


@pytest.mark.parametrize("method,way", [(1, 1), (2, 1), (2, 2)])
def test_fixed_step_scheme_fp64_bitwise(fq, oracle_lib, mono, method, way):
    # the 3/8 rule with Eq. step on the stretched grid (steps in cells of each
    # trial's start cell)
    B, grid = mono
    field = _field(fq, B, grid, pack=("f32", "f64", "gradb"))
    args = ((0.0, 0.0, 0.0), (63.0 / 61, 0, 0), (0, 55.0 / 43, 0), 61, 43)
    kw = dict(method=method, gradb_way=way, scheme=1, step=3.0 if method == 1 else 4.0)
    g = _plane(fq, field, *args, precision="f64", **kw)
    r = oracle.plane(B.astype(np.float64), grid, *args,
                     oracle.params(method=method, way=way, scheme=1, step=kw["step"]))
    assert_bitwise(g, r)
    g32 = _plane(fq, field, *args, precision="f32", **kw)
    rel = q_rel(g32, r)
    assert np.median(rel[np.isfinite(rel)]) < 1e-3
    if method == 1:
        seeds = np.random.default_rng(5).uniform([0, 0, 0], [63, 55, 31], size=(200, 3))
        g = to_np(fq.twist(field, torch.from_numpy(seeds).cuda(), fq.params(precision="f64", scheme=1, step=1.1)))
        field.check()
        assert_bitwise(g, oracle.twist(B.astype(np.float64), grid, seeds, oracle.params(scheme=1, step=1.1)))


def test_unsupported_modes(fq, mono):
    B, grid = mono
    field = _field(fq, B, grid)
    args = ((0.0, 0.0, 0.0), (1.0, 0, 0), (0, 1.0, 0), 4, 4)
    # Method II way 1 needs the gradient grid (not packed here); the step tape
    # is defined on stretched grids (tested below)
    for kw in (dict(method=2, gradb_way=1),):
        with pytest.raises(fq.FqslError) as ei:
            fq.qmap_plane(field, *args, fq.params(**kw))
        assert ei.value.status == 5, kw
    with pytest.raises(fq.FqslError) as ei:
        fq.Batch([field], [dict(origin=args[0], u=args[1], v=args[2], nu=4, nv=4)], fq.params())
    assert ei.value.status == 5


def test_full_size_stretched_workload_sampled(fq, oracle_lib):
    """The stretched benchmark workload at full size (the 256x256x128 monopole
    field on a stretched grid, 1024x1024 seeds on z=0) in the benchmark's
    launch configuration; the oracle recomputes a seeded sample of seeds."""
    B, grid, _ = synth.monopole24_stretched()
    field = _field(fq, B, grid)
    n = 1024
    args = ((0.0, 0.0, 0.0), (255.0 / n, 0, 0), (0, 255.0 / n, 0), n, n)
    g64 = _plane(fq, field, *args, precision="f64")
    g32 = _plane(fq, field, *args, precision="f32")
    sample = np.sort(np.random.default_rng(12).choice(n * n, 2000, replace=False))
    r = oracle.plane(B.astype(np.float64), grid, *args, oracle.params(), sample=sample)
    gs = {k: v[sample] for k, v in g64.items()}
    assert_fp64_parity(gs, r)
    assert_bitwise(gs, r)
    g32s = {k: v[sample] for k, v in g32.items()}
    assert np.mean(g32s["face2"] == r["face2"]) > 0.98
    rel = q_rel(g32s, r)
    assert np.median(rel[np.isfinite(rel)]) < 1e-3


def test_edge_cases_bitwise(fq, oracle_lib):
    # closed loops hit max_steps, a zero field is NULL_B, a plane partly outside
    # the box gives OUTSIDE and MIXED seeds, the tilted field rotates S0 (Q = 2):
    # every record as the oracle's, on a stretched grid
    g = synth.stretched_grid((24, 20, 16), (-1.0, -1.0, 0.0), (1.0, 1.0, 1.0), ratios=(1.05, 1.04, 1.08))
    cases = [
        ("loops", ((-0.5, -0.5, 0.5), (0.25, 0, 0), (0, 0.25, 0), 4, 4), dict(max_steps=3000, tol=1e-6)),
        ("zero", ((-0.5, -0.5, 0.0), (0.25, 0, 0), (0, 0.25, 0), 4, 4), {}),
        ("uniform", ((0.8, -0.2, 0.0), (0.2, 0, 0), (0, 0.2, 0), 4, 2), {}),
        ("tilted", ((-0.8, -0.8, 0.5), (0.1, 0, 0), (0, 0.1, 0), 16, 16), dict(tol=1e-10)),
    ]
    for kind, plane, kw in cases:
        B = synth.analytic_cube(kind, g)
        field = _field(fq, B, g)
        gg = _plane(fq, field, *plane, precision="f64", **kw)
        r = oracle.plane(B, g, *plane, oracle.params(**kw))
        assert_bitwise(gg, r)
        if kind == "loops":
            assert np.all(gg["status"] & oracle.MAXSTEPS)
        if kind == "zero":
            assert np.all(gg["status"] == oracle.NULL_B)
        if kind == "uniform":
            assert (gg["status"] & oracle.OUTSIDE).any() and (gg["status"] & oracle.MIXED).any()
        if kind == "tilted":
            assert np.all(gg["status"] & oracle.ROTATED)
            np.testing.assert_allclose(gg["Q"], 2.0, rtol=1e-8)
        field.close()


def test_strongly_stretched_axes_bitwise(fq, oracle_lib):
    # cell widths spanning a factor of about 800 along z and 60 along x: the
    # buckets (at most 16 per cell) then hold several nodes, so the cell search
    # often walks from the bucket's cell; the FP64 map stays the oracle's
    g = synth.RectGrid((synth.stretched_axis(40, 0.0, 39.0, 1.23, "edges"),
                        synth.stretched_axis(24, 0.0, 23.0, 1.0, "bottom"),
                        synth.stretched_axis(32, 0.0, 31.0, 1.25, "bottom")))
    w = [np.diff(g.axis(a)) for a in range(3)]
    assert w[0].max() / w[0].min() > 50 and w[2].max() / w[2].min() > 500
    ch = synth.random_charges(np.random.default_rng(8), 8, ((0.0, 39.0), (0.0, 23.0)), depth=(3.0, 8.0))
    B = synth.monopole_cube(g, ch, dtype=np.float32)
    field = _field(fq, B, g)
    args = ((0.0, 0.0, 0.0), (39.0 / 50, 0, 0), (0, 23.0 / 30, 0), 50, 30)
    gg = _plane(fq, field, *args, precision="f64")
    r = oracle.plane(B.astype(np.float64), g, *args, oracle.params())
    assert np.isfinite(r["Q"]).sum() > 1000
    assert_bitwise(gg, r)
    g32 = _plane(fq, field, *args, precision="f32")
    assert np.array_equal(g32["status"] & oracle.BAD, r["status"] & oracle.BAD)
    rel = q_rel(g32, r)
    assert np.median(rel[np.isfinite(rel)]) < 1e-3


# ---------------------------------------------------------------------------
# The discrete adjoint on a stretched grid (reading R16 under the frozen step
# sequence of R13): each step's start-cell widths held fixed, Eq. w0 weights
# in physical coordinates, the non-uniform three-point curl stencils; against
# the adjoint oracle's stretched replay (oracle/adjoint.py)
# ---------------------------------------------------------------------------
ADJ_N = (24, 22, 16)
ADJ_HI = (ADJ_N[0] - 1.0, ADJ_N[1] - 1.0, ADJ_N[2] - 1.0)
ADJ_Z0 = ((0.0, 0.0, 0.0), (ADJ_HI[0] / 12, 0.0, 0.0), (0.0, ADJ_HI[1] / 12, 0.0), 12, 12)
# an interior xz plane: seeds where |By/B| < 0.05 rotate S0
ADJ_XZ = ((0.0, ADJ_HI[1] * 0.41, 0.0), (ADJ_HI[0] / 14, 0.0, 0.0), (0.0, 0.0, ADJ_HI[2] / 9), 14, 9)


@pytest.fixture(scope="module")
def adj_mono():
    grid = synth.stretched_grid(ADJ_N, (0.0, 0.0, 0.0), ADJ_HI, (1.03, 1.02, 1.05))
    ch = synth.random_charges(np.random.default_rng(5), 6, ((0.0, ADJ_HI[0]), (0.0, ADJ_HI[1])), depth=(2.0, 5.0))
    return synth.monopole_cube(grid, ch, dtype=np.float64), grid


def _gpu_grad(fq, B, grid, plane, wq, wt, dtype=torch.float64, **kw):
    field = _field(fq, B, grid)
    t = fq.Tape()
    out = fq.qmap_plane(field, *plane, fq.params(tape=1, **kw), tape=t)
    st = out["status"].cpu().numpy()
    dB = fq.backward(field, torch.from_numpy(wq).cuda(), torch.from_numpy(wt).cuda(), dtype=dtype, tape=t)
    field.check()
    g = dB.cpu().numpy().astype(np.float64)
    t.close()
    return g, st, field


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("plane", [ADJ_Z0, ADJ_XZ], ids=["z0_plane", "interior_xz_plane"])
def test_stretched_fp64_gradient_matches_oracle_adjoint(fq, oracle_lib, adj_mono, plane):
    adj = pytest.importorskip("oracle.adjoint")
    B, grid = adj_mono
    m = plane[3] * plane[4]
    rng = np.random.default_rng(13)
    wq, wt = rng.standard_normal(m), rng.standard_normal(m)
    g, st, _ = _gpu_grad(fq, B, grid, plane, wq, wt, precision="f64")
    ref, log = adj.vjp(B, grid, *plane, wq, wt, oracle.params())
    assert np.array_equal(st & oracle.BAD, log["status"] & oracle.BAD)
    assert np.linalg.norm(ref) > 0
    assert _rel(g, ref) < 1e-10
    assert np.abs(g - ref).max() < 1e-10 * np.abs(ref).max()
    if plane is ADJ_XZ:
        assert (st & fq.LINE_ROTATED).sum() > 0


def test_stretched_rotated_seeds_gradient_matches_oracle(fq, oracle_lib, adj_mono):
    # weights on the usable rotated seeds only: the extra lines, their seed
    # adjoints and the frame VJP carry the whole gradient
    adj = pytest.importorskip("oracle.adjoint")
    B, grid = adj_mono
    ref_map = oracle.plane(B, grid, *ADJ_XZ, oracle.params())
    rot = ((ref_map["status"] & oracle.ROTATED) != 0) & np.isfinite(ref_map["Q"])
    assert rot.sum() >= 3
    wq = np.where(rot, 1.0 / np.where(rot, ref_map["Q"], 1.0), 0.0)
    g, _, _ = _gpu_grad(fq, B, grid, ADJ_XZ, wq, 0.0 * wq, precision="f64")
    ref, _ = adj.vjp(B, grid, *ADJ_XZ, wq, 0.0 * wq, oracle.params())
    assert np.linalg.norm(ref) > 0
    assert _rel(g, ref) < 1e-10


def test_stretched_fp64_tape_is_the_oracle_step_sequence(fq, oracle_lib, adj_mono):
    adj = pytest.importorskip("oracle.adjoint")
    B, grid = adj_mono
    field = _field(fq, B, grid)
    t = fq.Tape()
    fq.qmap_plane(field, *ADJ_Z0, fq.params(precision="f64", tape=1), tape=t)
    m = ADJ_Z0[3] * ADJ_Z0[4]
    ex = {k: v.cpu().numpy() for k, v in fq.tape_export(field, m, cap=2048, tape=t).items()}
    log = adj.lattice_log(B, grid, *ADJ_Z0, oracle.params())
    code, hh = adj.half_lines(log)
    for hl in range(2 * m):
        c = code[hl][code[hl] >= 0]
        if (log["status"][hl // 2] & oracle.BAD) != 0:
            assert ex["nsteps"][hl] == 0 and ex["code"][hl] == -1
            continue
        n = int(ex["nsteps"][hl])
        assert n == len(c) - 1 and np.all(c[:-1] == 0)
        assert ex["code"][hl] == c[-1]
        assert np.array_equal(ex["h"][hl, :n], hh[hl, :n])
    t.close()


@pytest.mark.parametrize("precision", ["f64", "f32", "f32acc64"])
def test_stretched_gradient_orthogonal_to_B(fq, oracle_lib, adj_mono, precision):
    # B -> c B leaves the frozen-sequence map unchanged, so <J^T w, B> = 0
    B, grid = adj_mono
    m = ADJ_Z0[3] * ADJ_Z0[4]
    rng = np.random.default_rng(17)
    g, _, _ = _gpu_grad(fq, B, grid, ADJ_Z0, rng.standard_normal(m), rng.standard_normal(m), precision=precision)
    tol = 1e-11 if precision == "f64" else 1e-4
    assert abs(np.sum(g * B)) < tol * np.linalg.norm(g) * np.linalg.norm(B)


def test_stretched_fp32_gradient_against_oracle(fq, oracle_lib, adj_mono):
    # the FP32 tracer takes its own step sequence (its controller amplifies
    # rounding), and the frozen-sequence derivative follows it: the bound is
    # stated, as on uniform grids
    adj = pytest.importorskip("oracle.adjoint")
    B, grid = adj_mono
    m = ADJ_Z0[3] * ADJ_Z0[4]
    rng = np.random.default_rng(19)
    wq, wt = rng.standard_normal(m), rng.standard_normal(m)
    g, _, _ = _gpu_grad(fq, B, grid, ADJ_Z0, wq, wt, dtype=torch.float32, precision="f32")
    ref, _ = adj.vjp(B, grid, *ADJ_Z0, wq, wt, oracle.params())
    assert _rel(g, ref) < 0.25


def test_stretched_hyperbolic_closed_form(fq):
    # B = (x, -y, 1) on a stretched grid over [-1, 1]^2 x [0, 1]: Q = e^2 + e^-2
    # on top exits and dQ/da = 2 (e^2 - e^-2) along dB = (x, -y, 0)
    grid = synth.stretched_grid((33, 33, 17), (-1.0, -1.0, 0.0), (1.0, 1.0, 1.0), (1.04, 1.04, 1.06))
    B = synth.analytic_cube("hyperbolic", grid)
    x, y, z = (np.asarray(c) for c in grid.coords)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    dB = np.stack([X, -Y, 0 * X], -1)
    plane = ((-0.3, -0.3, 0.0), (0.1, 0.0, 0.0), (0.0, 0.1, 0.0), 6, 6)
    w = np.random.default_rng(3).uniform(0.5, 1.5, 36)
    g, st, _ = _gpu_grad(fq, B, grid, plane, w, 0 * w, precision="f64", tol=1e-10)
    assert np.all(st & fq.LINE_BAD == 0)
    closed = 2.0 * (math.exp(2.0) - math.exp(-2.0))
    np.testing.assert_allclose(np.sum(g * dB), np.sum(w) * closed, rtol=1e-6)


def test_stretched_tape_refusals(fq, adj_mono):
    B, grid = adj_mono
    field = _field(fq, B, grid)
    for kw in (dict(precision="f64", reverse_precision="f32"), dict(precision="f32", reverse_precision="f64")):
        with pytest.raises(fq.FqslError) as ei:
            fq.qmap_plane(field, *ADJ_Z0, fq.params(tape=1, **kw), tape=fq.Tape())
        assert ei.value.status == 5


@pytest.mark.parametrize("plane", [ADJ_Z0, ADJ_XZ], ids=["z0_plane", "interior_xz_plane"])
def test_stretched_fixed_step_fp64_gradient_matches_oracle(fq, oracle_lib, adj_mono, plane):
    # the fixed-step 3/8 rule (Sec. 2.3, Eq. step) on the stretched grid: steps
    # in cells of each trial's start cell, the step of each line frozen
    adj = pytest.importorskip("oracle.adjoint")
    B, grid = adj_mono
    m = plane[3] * plane[4]
    rng = np.random.default_rng(23)
    wq, wt = rng.standard_normal(m), rng.standard_normal(m)
    kw = dict(scheme=1, step=0.3, step_min=0.05, max_steps=10 ** 6)
    g, st, _ = _gpu_grad(fq, B, grid, plane, wq, wt, precision="f64", **kw)
    ref, log = adj.vjp(B, grid, *plane, wq, wt, oracle.params(**kw))
    assert np.array_equal(st & oracle.BAD, log["status"] & oracle.BAD)
    assert np.linalg.norm(ref) > 0
    assert _rel(g, ref) < 1e-10
