"""The CUDA adjoint (fqsl_backward) against the FP64 CPU adjoint oracle
(oracle/adjoint.py) on the same seeded inputs, through the C ABI.

The derivative is that of the traced computation with each line's accepted
step sizes and exit kinds frozen. The FP64 tracer takes exactly the oracle's
steps (its forward is bit-identical), so its gradient must match the oracle's
to rounding; the FP32 tracer takes its own steps in float, and its gradient is
compared with a stated relative bound."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
adj = pytest.importorskip("oracle.adjoint")
pytestmark = pytest.mark.gpu

SMALL = dict(n=(24, 24, 24), count=6, radius_cells=4.0, dtype=np.float64)
PLANE16 = ((0.0, 0.0, 0.0), (23.0 / 16, 0.0, 0.0), (0.0, 23.0 / 16, 0.0), 16, 16)
# an interior xz plane: 21 seeds rotate S0 (their Q comes from four extra
# lines seeded along the frame of B at the seed, differentiated through it)
XZ = ((0.0, 18.3, 0.0), (23.0 / 20, 0.0, 0.0), (0.0, 0.0, 23.0 / 12), 20, 12)
PATCH = ((-0.3, -0.3, 0.0), (0.1, 0.0, 0.0), (0.0, 0.1, 0.0), 6, 6)


@pytest.fixture(scope="module")
def fq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_12569_gb300 as m

    return m


@pytest.fixture(scope="module")
def small():
    B, Bt, grid = synth.adjoint_cubes(**SMALL)
    return B, Bt, grid


def _field(fq, B, grid):
    return fq.Field(torch.from_numpy(np.ascontiguousarray(B)).cuda(), grid.origin, grid.spacing)


def _weights(seed, m):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(m), rng.standard_normal(m)


def _gpu_vjp(fq, field, plane, wq, wt, dtype=torch.float64, **kw):
    out = fq.qmap_plane(field, *plane, fq.params(tape=1, **kw))
    st = out["status"].cpu().numpy()
    dB = fq.backward(field, torch.from_numpy(wq).cuda(), torch.from_numpy(wt).cuda(), dtype=dtype)
    field.check()
    return dB.cpu().numpy().astype(np.float64), st


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("plane", [PLANE16, XZ], ids=["z0_plane", "interior_xz_plane"])
def test_fp64_gradient_matches_oracle_adjoint(fq, small, plane):
    B, _, grid = small
    field = _field(fq, B, grid)
    m = plane[3] * plane[4]
    wq, wt = _weights(11, m)
    g, st = _gpu_vjp(fq, field, plane, wq, wt, precision="f64")
    ref, log = adj.vjp(B, grid, *plane, wq, wt, oracle.params())
    assert np.array_equal(st & oracle.BAD, log["status"] & oracle.BAD)
    assert np.linalg.norm(ref) > 0
    assert _rel(g, ref) < 1e-10
    assert np.abs(g - ref).max() < 1e-10 * np.abs(ref).max()
    if plane is XZ:
        assert (st & fq.LINE_ROTATED).any()


def _rotated_weights(fq, field, B, grid):
    # log-Q weights on the usable rotated seeds of XZ only
    ref = oracle.plane(B, grid, *XZ, oracle.params())
    rot = ((ref["status"] & oracle.ROTATED) != 0) & np.isfinite(ref["Q"])
    assert rot.sum() >= 15
    wq = np.where(rot, 1.0 / np.where(rot, ref["Q"], 1.0), 0.0)
    return wq, 0.0 * wq


def test_rotated_seeds_gradient_matches_oracle(fq, small):
    # only rotated seeds weighted: the extra lines' reverse sweep, their seed
    # adjoints and the frame VJP carry the whole gradient
    B, _, grid = small
    field = _field(fq, B, grid)
    wq, wt = _rotated_weights(fq, field, B, grid)
    g, st = _gpu_vjp(fq, field, XZ, wq, wt, precision="f64")
    ref, _ = adj.vjp(B, grid, *XZ, wq, wt, oracle.params())
    assert np.linalg.norm(ref) > 0
    assert _rel(g, ref) < 1e-10
    # FP32 reverse sweep on the same (oracle) steps
    g32, _ = _gpu_vjp(fq, field, XZ, wq, wt, dtype=torch.float32, precision="f64", reverse_precision="f32")
    assert _rel(g32, ref) < 2e-3


def test_rotated_frame_is_differentiated(fq, small, monkeypatch):
    # Planted in the oracle: with the frame of the extra seeds held constant
    # (no derivative through B at the seed) the oracle's gradient moves away
    # from the CUDA one by far more than rounding.
    B, _, grid = small
    field = _field(fq, B, grid)
    wq, wt = _rotated_weights(fq, field, B, grid)
    g, _ = _gpu_vjp(fq, field, XZ, wq, wt, precision="f64")
    real = adj.perp_frame_t
    monkeypatch.setattr(adj, "perp_frame_t", lambda bh, m: tuple(x.detach() for x in real(bh.detach(), m)))
    planted, _ = adj.vjp(B, grid, *XZ, wq, wt, oracle.params())
    assert _rel(g, planted) > 1e-3


def test_rotated_seeds_survive_an_untaped_map(fq, small):
    # the rotated-seed count of a taped map is kept with its tape: an untaped
    # map on the same field in between leaves the gradient unchanged
    B, _, grid = small
    field = _field(fq, B, grid)
    m = XZ[3] * XZ[4]
    wq, wt = _weights(13, m)
    g0, _ = _gpu_vjp(fq, field, XZ, wq, wt, precision="f64")
    fq.qmap_plane(field, *XZ, fq.params(precision="f64", tape=1))
    fq.qmap_plane(field, *PLANE16, fq.params(precision="f64"))
    fq.qmap_plane(field, (0.0, 4.3, 0.0), (23.0 / 8, 0.0, 0.0), (0.0, 0.0, 23.0 / 8), 8, 8, fq.params())
    g1 = fq.backward(field, torch.from_numpy(wq).cuda(), torch.from_numpy(wt).cuda(), dtype=torch.float64)
    field.check()
    # (node sums are accumulated with atomics: equal up to their order)
    assert _rel(g1.cpu().numpy(), g0) < 1e-13


@pytest.mark.parametrize("reverse,bound", [("f32", 2e-3), ("f32acc64", 2e-3)])
def test_fp32_reverse_sweep_on_the_oracle_steps(fq, small, reverse, bound):
    # FP64 taped forward (the oracle's own step sequence), reverse sweep in
    # float: isolates the float arithmetic of the reverse sweep
    B, _, grid = small
    field = _field(fq, B, grid)
    m = PLANE16[3] * PLANE16[4]
    wq, wt = _weights(12, m)
    g, st = _gpu_vjp(fq, field, PLANE16, wq, wt, dtype=torch.float32, precision="f64", reverse_precision=reverse)
    ref, _ = adj.vjp(B, grid, *PLANE16, wq, wt, oracle.params())
    assert _rel(g, ref) < bound


@pytest.mark.parametrize("precision", ["f32", "f32acc64"])
def test_fp32_forward_gradient_against_oracle(fq, small, precision):
    # The FP32 tracer takes its own step sequence (the controller amplifies
    # rounding differences), and the frozen-sequence gradient depends on where
    # the stage points fall: even FP64 with tol x (1 + 1e-6) moves node-level
    # gradients by a few percent. Stated bound on the node-level relative
    # error for log-Q and Tw weights (the loss's form).
    B, _, grid = small
    B32 = B.astype(np.float32)
    field = _field(fq, B32, grid)
    m = PLANE16[3] * PLANE16[4]
    wq, wt = _weights(12, m)
    Qo = oracle.plane(B32.astype(np.float64), grid, *PLANE16, oracle.params())["Q"]
    wq = wq / np.where(np.isfinite(Qo), Qo, 1.0)
    g, st = _gpu_vjp(fq, field, PLANE16, wq, wt, dtype=torch.float32, precision=precision)
    ref, _ = adj.vjp(B32.astype(np.float64), grid, *PLANE16, wq, wt, oracle.params())
    assert _rel(g, ref) < 0.25


def test_fp64_tape_is_the_oracle_step_sequence(fq, small):
    # the FP64 tracer's recorded steps are the oracle's, bit for bit
    B, _, grid = small
    field = _field(fq, B, grid)
    p = fq.params(precision="f64", tape=1)
    fq.qmap_plane(field, *PLANE16, p)
    m = PLANE16[3] * PLANE16[4]
    t = {k: v.cpu().numpy() for k, v in fq.tape_export(field, m, cap=2048).items()}
    log = adj.lattice_log(B, grid, *PLANE16, oracle.params())
    code, hh = adj.half_lines(log)
    for hl in range(2 * m):
        c = code[hl][code[hl] >= 0]
        good = (log["status"][hl // 2] & oracle.BAD) == 0
        if not good:
            assert t["nsteps"][hl] == 0 and t["code"][hl] == -1
            continue
        n = int(t["nsteps"][hl])
        assert n == len(c) - 1 and np.all(c[:-1] == 0)
        assert t["code"][hl] == c[-1]
        assert np.array_equal(t["h"][hl, :n], hh[hl, :n])
        if c[-1] >= adj.CHORD:
            assert t["hx"][hl] == hh[hl, n]


def test_dot_product_with_oracle_tangent_mode(fq, small):
    # <J v, w> from the oracle's forward-mode derivative = <v, J^T w> from the GPU
    B, _, grid = small
    field = _field(fq, B, grid)
    m = PLANE16[3] * PLANE16[4]
    wq, wt = _weights(13, m)
    v = np.random.default_rng(14).standard_normal(B.shape)
    g, st = _gpu_vjp(fq, field, PLANE16, wq, wt, precision="f64")
    dQ, dTw, us, log = adj.jvp(B, grid, *PLANE16, v, oracle.params())
    good = (log["status"] & oracle.BAD) == 0
    lhs = np.sum(wq[us] * dQ[us]) + np.sum(wt[good] * dTw[good])
    rhs = np.sum(v * g)
    assert abs(lhs - rhs) < 1e-10 * (abs(lhs) + 1e-3 * np.linalg.norm(g) * np.linalg.norm(v))


@pytest.mark.parametrize("precision,tol", [("f64", 1e-11), ("f32", 1e-4)])
def test_gradient_orthogonal_to_B(fq, small, precision, tol):
    # the map is invariant under B -> c B, so <J^T w, B> = 0
    B, _, grid = small
    Bp = B if precision == "f64" else B.astype(np.float32)
    field = _field(fq, Bp, grid)
    m = PLANE16[3] * PLANE16[4]
    wq, wt = _weights(15, m)
    g, _ = _gpu_vjp(fq, field, PLANE16, wq, wt, precision=precision)
    Bd = Bp.astype(np.float64)
    assert abs(np.sum(g * Bd)) < tol * np.linalg.norm(g) * np.linalg.norm(Bd)


def _mesh(grid):
    x, y, z = (grid.axis(a) for a in range(3))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


@pytest.mark.parametrize("precision,rtol", [("f64", 1e-5), ("f32", 1e-3)])
def test_hyperbolic_closed_form(fq, precision, rtol):
    # B = (x, -y, 1): sum_s w_s dQ_s/da along dB = (x, -y, 0) = sum w * 2L(e^2L - e^-2L)
    grid = synth.ANALYTIC_GRID
    B = synth.analytic_cube("hyperbolic", grid)
    field = _field(fq, B if precision == "f64" else B.astype(np.float32), grid)
    X, Y, Z = _mesh(grid)
    dB = np.stack([X, -Y, 0 * X], -1)
    w = np.random.default_rng(3).uniform(0.5, 1.5, 36)
    g, st = _gpu_vjp(fq, field, PATCH, w, 0 * w, precision=precision)
    assert not (st & (oracle.BAD | oracle.MIXED)).any()
    closed = 2.0 * (math.exp(2.0) - math.exp(-2.0))
    np.testing.assert_allclose(np.sum(g * dB), np.sum(w) * closed, rtol=rtol)


@pytest.mark.parametrize("precision,rtol", [("f64", 1e-3), ("f32", 2e-3)])
def test_rotation_closed_form(fq, precision, rtol):
    # B = (-q y, q x, 1): sum_s w_s dTw_s/dq along dB = (-y, x, 0)
    grid = synth.ANALYTIC_GRID
    q = 2.0 * math.pi
    B = synth.analytic_cube("rotation", grid, q=q)
    field = _field(fq, B if precision == "f64" else B.astype(np.float32), grid)
    X, Y, Z = _mesh(grid)
    dB = np.stack([-Y, X, 0 * X], -1)
    w = np.random.default_rng(4).uniform(0.5, 1.5, 36)
    g, _ = _gpu_vjp(fq, field, PATCH, 0 * w, w, precision=precision)
    r0 = np.asarray(grid.origin) + np.asarray(grid.spacing) * adj.seeds_index(grid, *PATCH)
    r2 = r0[:, 0] ** 2 + r0[:, 1] ** 2
    closed = (1.0 + q * q * r2) ** -1.5 / (2.0 * math.pi)
    np.testing.assert_allclose(np.sum(g * dB), np.sum(w * closed), rtol=rtol)


def test_checkpoint_interval_does_not_change_the_gradient(fq, small):
    B, _, grid = small
    field = _field(fq, B, grid)
    m = PLANE16[3] * PLANE16[4]
    wq, wt = _weights(16, m)
    gs = [_gpu_vjp(fq, field, PLANE16, wq, wt, precision="f64", tape_chunk=k)[0] for k in (1, 3, 16, 32)]
    for g in gs[1:]:
        assert _rel(g, gs[0]) < 1e-12


def test_tape_pool_grows_when_exhausted(fq, small):
    # tight tolerance and one step per chunk: the first pool guess is too small,
    # fqsl_backward traces the map again with a larger pool
    B, _, grid = small
    field = _field(fq, B, grid)
    m = PLANE16[3] * PLANE16[4]
    wq, wt = _weights(17, m)
    kw = dict(precision="f64", tol=1e-7, max_steps=1000000)
    g1, _ = _gpu_vjp(fq, field, PLANE16, wq, wt, tape_chunk=1, **kw)
    g16, _ = _gpu_vjp(fq, field, PLANE16, wq, wt, tape_chunk=16, **kw)
    assert _rel(g1, g16) < 1e-12
    ref, _ = adj.vjp(B, grid, *PLANE16, wq, wt, oracle.params(tol=1e-7, max_steps=1000000))
    assert _rel(g1, ref) < 1e-10


def test_kept_states_grow_to_the_map(fq, small):
    # one step per chunk: the first taped call keeps the states of two chunks
    # per direction, fewer than the map takes, so its backward recomputes them
    # from the checkpoints; the next taped call on the same tape keeps every
    # chunk the first one used. Both gradients equal the oracle adjoint.
    B, _, grid = small
    field = _field(fq, B, grid)
    m = PLANE16[3] * PLANE16[4]
    wq, wt = _weights(23, m)
    g1, _ = _gpu_vjp(fq, field, PLANE16, wq, wt, precision="f64", tape_chunk=1)
    g2, _ = _gpu_vjp(fq, field, PLANE16, wq, wt, precision="f64", tape_chunk=1)
    assert _rel(g2, g1) < 1e-12
    ref, _ = adj.vjp(B, grid, *PLANE16, wq, wt, oracle.params())
    assert _rel(g1, ref) < 1e-10 and _rel(g2, ref) < 1e-10


def test_loss_kernel_matches_oracle_loss(fq, small):
    B, Bt, grid = small
    field = _field(fq, B, grid)
    ftgt = _field(fq, Bt, grid)
    p = fq.params(precision="f64")
    out = fq.qmap_plane(field, *PLANE16, p)
    tgt = fq.qmap_plane(ftgt, *PLANE16, p)
    loss, dQ, dTw = fq.loss_logq_tw(out["Q"], out["Tw"], tgt["Q"], tgt["Tw"], out["status"], 0.1)
    Q = torch.tensor(out["Q"].cpu().numpy(), requires_grad=True)
    Tw = torch.tensor(out["Tw"].cpu().numpy(), requires_grad=True)
    st = out["status"].cpu().numpy()
    usable = torch.from_numpy((st & (oracle.BAD | oracle.MIXED)) == 0)
    ref, use = adj.log_q_tw_loss(Q, Tw, tgt["Q"].cpu().numpy(), tgt["Tw"].cpu().numpy(), usable, 0.1)
    ref.backward()
    assert int(use.sum()) > 200
    np.testing.assert_allclose(float(loss), float(ref.detach()), rtol=1e-12)
    np.testing.assert_allclose(dQ.cpu().numpy(), Q.grad.numpy(), rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(dTw.cpu().numpy(), Tw.grad.numpy(), rtol=1e-12, atol=1e-300)


def test_loss_in_place_buffers(fq, small):
    # dQ, dTw given as the Q and Tw inputs themselves (the kernel keeps its
    # log-Q differences in the output buffers only when they are not inputs):
    # the same loss and gradient as with separate buffers, bit for bit
    B, Bt, grid = small
    field = _field(fq, B, grid)
    ftgt = _field(fq, Bt, grid)
    p = fq.params(precision="f64")
    out = fq.qmap_plane(field, *PLANE16, p)
    tgt = fq.qmap_plane(ftgt, *PLANE16, p)
    loss, dQ, dTw = fq.loss_logq_tw(out["Q"], out["Tw"], tgt["Q"], tgt["Tw"], out["status"], 0.1)
    Qi, Twi = out["Q"].clone(), out["Tw"].clone()
    buf = dict(sums=torch.empty(2, dtype=torch.float64, device="cuda"),
               loss=torch.empty((), dtype=torch.float64, device="cuda"), dQ=Qi, dTw=Twi)
    loss2, dQ2, dTw2 = fq.loss_logq_tw(Qi, Twi, tgt["Q"], tgt["Tw"], out["status"], 0.1, out=buf)
    assert dQ2.data_ptr() == Qi.data_ptr()
    assert float(loss2) == float(loss)
    assert torch.equal(dQ2, dQ) and torch.equal(dTw2, dTw)
    assert int((dQ != 0).sum()) > 200


@pytest.mark.parametrize("plane", [PLANE16, XZ], ids=["z0_plane", "interior_xz_plane"])
def test_loss_gradient_end_to_end_matches_oracle(fq, small, plane):
    # loss -> dQ, dTw (loss kernel) -> dB (fqsl_backward), FP64, against the
    # oracle's autograd of the same loss over the frozen step sequence
    B, Bt, grid = small
    field = _field(fq, B, grid)
    tgt = oracle.plane(Bt, grid, *plane, oracle.params())
    p = fq.params(precision="f64", tape=1)
    out = fq.qmap_plane(field, *plane, p)
    qt = torch.from_numpy(tgt["Q"]).cuda()
    twt = torch.from_numpy(tgt["Tw"]).cuda()
    loss, dQ, dTw = fq.loss_logq_tw(out["Q"], out["Tw"], qt, twt, out["status"], 0.1)
    dB = fq.backward(field, dQ, dTw, dtype=torch.float64).cpu().numpy()
    ref_loss, ref_g, _ = adj.loss_grad(B, grid, *plane, tgt["Q"], tgt["Tw"], oracle.params())
    np.testing.assert_allclose(float(loss), ref_loss, rtol=1e-11)
    assert _rel(dB, ref_g) < 1e-10


def test_autograd_function(fq, small):
    B, Bt, grid = small
    Bd = torch.from_numpy(B).cuda()
    field = _field(fq, B, grid)
    tgt = oracle.plane(Bt, grid, *PLANE16, oracle.params())
    p = fq.params(precision="f64")
    Bv = Bd.clone().requires_grad_(True)
    Q, Tw = fq.QTwPlane.apply(Bv, field, *PLANE16, p)
    st = fq.qmap_plane(field, *PLANE16, p)["status"]
    loss, dQ, dTw = fq.loss_logq_tw(Q.detach(), Tw.detach(), torch.from_numpy(tgt["Q"]).cuda(),
                                    torch.from_numpy(tgt["Tw"]).cuda(), st, 0.1)
    torch.autograd.backward([Q, Tw], [dQ, dTw])
    _, ref_g, _ = adj.loss_grad(B, grid, *PLANE16, tgt["Q"], tgt["Tw"], oracle.params())
    assert Bv.grad is not None and Bv.grad.dtype == torch.float64
    assert _rel(Bv.grad.cpu().numpy(), ref_g) < 1e-10


def test_backward_argument_errors(fq, small):
    import ctypes as C

    from paper_2208_12569_gb300 import fqsl as raw

    B, _, grid = small
    field = _field(fq, B, grid)
    with pytest.raises(RuntimeError, match="no taped map"):
        fq.backward(field, None, None)
    dB = torch.zeros(B.shape, dtype=torch.float64, device="cuda")
    assert raw._lib.fqsl_backward(field.handle, None, None, None, C.c_void_p(dB.data_ptr()), fq.F64, None) == 1
    assert b"NULL tape" in raw._lib.fqsl_last_error()
    # params.tape = 1 needs somewhere to put the tape
    p = fq.params(tape=1)
    out = fq.alloc_out(PLANE16[3] * PLANE16[4])
    assert raw._lib.fqsl_qmap_plane(field.handle, raw._vec3(PLANE16[0]), raw._vec3(PLANE16[1]),
                                    raw._vec3(PLANE16[2]), PLANE16[3], PLANE16[4], C.byref(p),
                                    C.byref(raw._out_struct(out)), None, None) == 1
    assert b"tape_or_null" in raw._lib.fqsl_last_error()
    with pytest.raises(fq.FqslError) as ei:
        fq.qmap_plane(field, *PLANE16, fq.params(tape=1, method=2))
    assert ei.value.status == 5
    with pytest.raises(fq.FqslError) as ei:
        fq.qmap_volume(field, (0.0, 0.0, 0.0), (2.0, 2.0, 2.0), 4, 4, 4, fq.params(tape=1, method=2))
    assert ei.value.status == 5
    with pytest.raises(fq.FqslError) as ei:
        fq.qmap_plane(field, *PLANE16, fq.params(tape=1, tape_chunk=33))
    assert ei.value.status == 1
    # zero weights give a zero gradient
    fq.qmap_plane(field, *PLANE16, fq.params(tape=1))
    dB = fq.backward(field, None, None)
    field.check()
    assert float(dB.abs().max()) == 0.0


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("plane", [PLANE16, XZ], ids=["z0_plane", "interior_xz_plane"])
def test_taped_map_equals_plain_map(fq, small, precision, plane):
    # the taped tracer runs the two directions of a line as separate items;
    # the map it returns is the plain map's
    from parity import assert_bitwise, to_np

    B, _, grid = small
    field = _field(fq, B, grid)
    plain = to_np(fq.qmap_plane(field, *plane, fq.params(precision=precision)))
    taped = to_np(fq.qmap_plane(field, *plane, fq.params(precision=precision, tape=1)))
    field.check()
    if precision == "f64":
        assert_bitwise(taped, plain)
    else:
        for k in ("face1", "face2", "status", "steps"):
            assert np.array_equal(taped[k], plain[k]), k
        ok = np.isfinite(plain["Q"])
        assert np.array_equal(ok, np.isfinite(taped["Q"]))
        np.testing.assert_allclose(taped["Q"][ok], plain["Q"][ok], rtol=1e-5)
        np.testing.assert_allclose(taped["Tw"], plain["Tw"], rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("scheme", [0, 1], ids=["rkf45", "fixed_step"])
def test_volume_gradient_matches_oracle(fq, small, scheme):
    # a volume map: each z-layer is its own S0, so its adjoint is the sum of
    # the layers' plane adjoints (scheme 1: the 3/8 rule with Eq. step)
    B, _, grid = small
    field = _field(fq, B, grid)
    step = (23.0 / 6, 23.0 / 6, 4.0)
    nx, ny, nz = 6, 6, 3
    m = nx * ny * nz
    wq, wt = _weights(21, m)
    kw = dict(scheme=1, step=0.3, step_min=0.05, max_steps=10 ** 6) if scheme else {}
    out = fq.qmap_volume(field, (0.0, 0.0, 0.0), step, nx, ny, nz, fq.params(precision="f64", tape=1, **kw))
    st = out["status"].cpu().numpy()
    dB = fq.backward(field, torch.from_numpy(wq).cuda(), torch.from_numpy(wt).cuda(), dtype=torch.float64)
    field.check()
    g = dB.cpu().numpy()
    ref = np.zeros_like(B)
    per = nx * ny
    for k in range(nz):
        plane = ((0.0, 0.0, (k + 0.5) * step[2]), (step[0], 0.0, 0.0), (0.0, step[1], 0.0), nx, ny)
        r, log = adj.vjp(B, grid, *plane, wq[k * per:(k + 1) * per], wt[k * per:(k + 1) * per],
                         oracle.params(**kw))
        line_bits = oracle.BAD | oracle.ROTATED | oracle.CHORD | oracle.STALL
        assert np.array_equal(log["status"] & line_bits, st[k * per:(k + 1) * per] & line_bits)
        ref += r
    assert np.linalg.norm(ref) > 0
    assert _rel(g, ref) < 1e-10


def test_backward_refuses_a_stale_tape(fq, small):
    B, _, grid = small
    field = _field(fq, B, grid)
    t = fq.Tape()
    fq.qmap_plane(field, *PLANE16, fq.params(tape=1), tape=t)
    fq.qmap_plane(field, *PLANE16, fq.params())  # an untaped map leaves the tape alone
    fq.backward(field, None, None, tape=t)
    field.check()
    field.update(torch.from_numpy(B).cuda())
    with pytest.raises(fq.FqslError) as ei:
        fq.backward(field, None, None, tape=t)
    assert ei.value.status == 1 and "updated" in str(ei.value)
    # a tape recorded on another field is refused
    other = _field(fq, B, grid)
    t2 = fq.Tape()
    fq.qmap_plane(other, *PLANE16, fq.params(tape=1), tape=t2)
    with pytest.raises(fq.FqslError) as ei:
        fq.backward(field, None, None, tape=t2)
    assert ei.value.status == 1 and "another field" in str(ei.value)
    # a tape outlives its field for export (and is released on its own)
    other.close()
    ex = fq.tape_export(None, PLANE16[3] * PLANE16[4], cap=0, tape=t2)
    assert int(ex["nsteps"].sum()) > 0
    t.close()
    t2.close()


def test_two_taped_maps_on_one_field(fq, small):
    """Two taped maps of one field held at once in their own tapes (Q on two
    planes in one loss): each backward, taken in reverse order, gives that
    map's FP64 gradient equal to the oracle adjoint; an untaped map, a third
    taped map in another tape and the first backward in between change nothing."""
    B, _, grid = small
    field = _field(fq, B, grid)
    w = {}
    tapes = {}
    for name, plane, seed in (("z0", PLANE16, 31), ("xz", XZ, 32)):
        w[name] = _weights(seed, plane[3] * plane[4])
        tapes[name] = fq.Tape()
        fq.qmap_plane(field, *plane, fq.params(precision="f64", tape=1), tape=tapes[name])
    fq.qmap_plane(field, *PATCH, fq.params(precision="f64"))
    t3 = fq.Tape()
    fq.qmap_plane(field, *PATCH, fq.params(precision="f32", tape=1), tape=t3)
    grads = {}
    for name in ("xz", "z0"):
        wq, wt = w[name]
        dB = fq.backward(field, torch.from_numpy(wq).cuda(), torch.from_numpy(wt).cuda(), dtype=torch.float64,
                         tape=tapes[name])
        field.check()
        grads[name] = dB.cpu().numpy()
    for name, plane in (("z0", PLANE16), ("xz", XZ)):
        ref, _ = adj.vjp(B, grid, *plane, *w[name], oracle.params())
        assert np.linalg.norm(ref) > 0
        assert _rel(grads[name], ref) < 1e-10, name
    # the same weights again on the same tape: the same gradient
    wq, wt = w["z0"]
    again = fq.backward(field, torch.from_numpy(wq).cuda(), torch.from_numpy(wt).cuda(), dtype=torch.float64,
                        tape=tapes["z0"]).cpu().numpy()
    assert _rel(again, grads["z0"]) < 1e-13
    for t in (*tapes.values(), t3):
        t.close()


def test_autograd_reuses_released_tapes(fq, small):
    # a QTwPlane forward whose graph was released hands its tape back to the
    # field: a training loop reuses one tape (and its device memory)
    import gc

    B, _, grid = small
    field = _field(fq, B, grid)
    Bv = torch.from_numpy(B).cuda().requires_grad_(True)
    handles = set()
    for _ in range(3):
        Q, Tw = fq.QTwPlane.apply(Bv, field, *PLANE16, fq.params(precision="f64"))
        torch.autograd.backward([Q], [torch.ones_like(Q)])
        del Q, Tw
        gc.collect()
        assert len(field._free_tapes) == 1
        handles.add(field._free_tapes[0].value)
    assert len(handles) == 1
    field.close()
    assert field._free_tapes == []


def test_autograd_two_planes_in_one_loss(fq, small):
    # QTwPlane keeps its own tape: Q on two planes of one field in one graph
    B, _, grid = small
    field = _field(fq, B, grid)
    p = fq.params(precision="f64")
    Bv = torch.from_numpy(B).cuda().requires_grad_(True)
    (wq1, wt1), (wq2, wt2) = _weights(41, PLANE16[3] * PLANE16[4]), _weights(42, XZ[3] * XZ[4])
    Q1, Tw1 = fq.QTwPlane.apply(Bv, field, *PLANE16, p)
    Q2, Tw2 = fq.QTwPlane.apply(Bv, field, *XZ, p)
    c = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    torch.autograd.backward([Q1, Tw1, Q2, Tw2], [c(wq1), c(wt1), c(wq2), c(wt2)])
    r1, _ = adj.vjp(B, grid, *PLANE16, wq1, wt1, oracle.params())
    r2, _ = adj.vjp(B, grid, *XZ, wq2, wt2, oracle.params())
    assert _rel(Bv.grad.cpu().numpy(), r1 + r2) < 1e-10


def test_full_size_workload_sampled(fq):
    # the differentiation workload at full size (128x128x64 cube, 256^2 seeds,
    # checkpoints every 16 steps, the launch the benchmark times): weights on a
    # seeded sample of 32 seeds, against the oracle traced for just those lines
    # and their neighbours
    B, _, grid = synth.adjoint_cubes(seed=2208, n=(128, 128, 64))
    plane = ((0.0, 0.0, 0.0), (127.0 / 256, 0.0, 0.0), (0.0, 127.0 / 256, 0.0), 256, 256)
    n = 256 * 256
    rng = np.random.default_rng(2208)
    sample = np.sort(rng.choice(n, 32, replace=False))
    wq, wt = rng.standard_normal(32), rng.standard_normal(32)
    WQ, WT = np.zeros(n), np.zeros(n)
    WQ[sample], WT[sample] = wq, wt
    ref, info = adj.vjp_sample(B.astype(np.float64), grid, *plane, sample, wq, wt, oracle.params())
    assert np.linalg.norm(ref) > 0
    field = _field(fq, B, grid)
    g64, _ = _gpu_vjp(fq, field, plane, WQ, WT, precision="f64", tape_chunk=16)
    assert _rel(g64, ref) < 1e-10
    g32r, _ = _gpu_vjp(fq, field, plane, WQ, WT, dtype=torch.float32, precision="f64", reverse_precision="f32",
                       tape_chunk=16)
    assert _rel(g32r, ref) < 2e-3
    g32, _ = _gpu_vjp(fq, field, plane, WQ, WT, dtype=torch.float32, precision="f32", tape_chunk=16)
    assert _rel(g32, ref) < 0.25
    Bd = B.astype(np.float64)
    for g in (g64, g32):
        assert abs(np.sum(g * Bd)) < 1e-4 * np.linalg.norm(g) * np.linalg.norm(Bd)


def test_fp32_loss_gradient_agrees_with_fp64_along_smooth_directions(fq):
    """The full-size differentiation workload's loss gradient in FP32 and in
    FP64: each follows its own step sequence, so node by node they differ
    (about 28 %), but along smooth directions (the field of a buried source
    pair) their directional derivatives agree to a few per cent."""
    B, Bt, grid = synth.adjoint_cubes(seed=2208, n=(128, 128, 64))
    plane = ((0.0, 0.0, 0.0), (127.0 / 256, 0.0, 0.0), (0.0, 127.0 / 256, 0.0), 256, 256)
    ftgt = _field(fq, Bt, grid)
    tgt = fq.qmap_plane(ftgt, *plane, fq.params(precision="f32"))
    field = _field(fq, B, grid)
    g = {}
    for prec in ("f32", "f64"):
        out = fq.qmap_plane(field, *plane, fq.params(precision=prec, tape=1))
        _, dQ, dTw = fq.loss_logq_tw(out["Q"], out["Tw"], tgt["Q"], tgt["Tw"], out["status"], 0.1)
        g[prec] = fq.backward(field, dQ, dTw, dtype=torch.float64).cpu().numpy()
        field.check()
    assert _rel(g["f32"], g["f64"]) > 0.05  # the node-level difference is real
    rng = np.random.default_rng(2219)
    B64 = B.astype(np.float64)
    for _ in range(4):
        ch = synth.random_charges(rng, 2, ((0.0, 127.0), (0.0, 127.0)), depth=(4.0, 16.0))
        dB = synth.monopole_cube(grid, ch, dtype=np.float64)
        dB *= np.sqrt(np.mean(B64 * B64) / np.mean(dB * dB))
        d32, d64 = float(np.sum(g["f32"] * dB)), float(np.sum(g["f64"] * dB))
        assert abs(d32 - d64) < 0.05 * abs(d64), (d32, d64)


# ---------------------------------------------------------------------------
# the fixed-step scheme (Sec. 2.3: Kutta's 3/8 rule with the per-line step of
# Sec. 4 Eq. step): the tape holds the fixed steps (grazing halvings
# included), the reverse sweep runs the four-stage step
# ---------------------------------------------------------------------------
FIXED = dict(scheme=1, step=0.3, step_min=0.05, max_steps=10 ** 6)


@pytest.mark.parametrize("plane", [PLANE16, XZ], ids=["z0_plane", "interior_xz_plane"])
def test_fixed_step_fp64_gradient_matches_oracle(fq, small, plane):
    B, _, grid = small
    field = _field(fq, B, grid)
    m = plane[3] * plane[4]
    wq, wt = _weights(21, m)
    g, st = _gpu_vjp(fq, field, plane, wq, wt, precision="f64", **FIXED)
    ref, log = adj.vjp(B, grid, *plane, wq, wt, oracle.params(**FIXED))
    assert log["scheme"] == 1
    assert np.array_equal(st & oracle.BAD, log["status"] & oracle.BAD)
    assert np.linalg.norm(ref) > 0
    assert _rel(g, ref) < 1e-10
    assert np.abs(g - ref).max() < 1e-10 * np.abs(ref).max()
    if plane is XZ:
        assert (st & fq.LINE_ROTATED).any()
    # the RKF45 gradient of the same map is a different vector
    g45, _ = _gpu_vjp(fq, field, plane, wq, wt, precision="f64")
    assert _rel(g45, ref) > 1e-6


def test_fixed_step_tape_is_the_oracle_step_sequence(fq, small):
    # every recorded step is the line's Eq. step value (or a grazing halving
    # of it), bit for bit the oracle's
    B, _, grid = small
    field = _field(fq, B, grid)
    fq.qmap_plane(field, *PLANE16, fq.params(precision="f64", tape=1, **FIXED))
    m = PLANE16[3] * PLANE16[4]
    t = {k: v.cpu().numpy() for k, v in fq.tape_export(field, m, cap=4096).items()}
    log = adj.lattice_log(B, grid, *PLANE16, oracle.params(**FIXED))
    code, hh = adj.half_lines(log)
    distinct = set()
    for hl in range(2 * m):
        c = code[hl][code[hl] >= 0]
        if (log["status"][hl // 2] & oracle.BAD) != 0:
            assert t["nsteps"][hl] == 0 and t["code"][hl] == -1
            continue
        n = int(t["nsteps"][hl])
        assert n == len(c) - 1 and t["code"][hl] == c[-1]
        assert np.array_equal(t["h"][hl, :n], hh[hl, :n])
        distinct.update(np.unique(t["h"][hl, :n]).tolist())
    assert len(distinct) > 50  # Eq. step gives each line its own step


@pytest.mark.parametrize("reverse", ["f32", "f32acc64"])
def test_fixed_step_fp32_reverse_sweep_on_the_oracle_steps(fq, small, reverse):
    B, _, grid = small
    field = _field(fq, B, grid)
    m = PLANE16[3] * PLANE16[4]
    wq, wt = _weights(22, m)
    g, _ = _gpu_vjp(fq, field, PLANE16, wq, wt, dtype=torch.float32, precision="f64", reverse_precision=reverse,
                    **FIXED)
    ref, _ = adj.vjp(B, grid, *PLANE16, wq, wt, oracle.params(**FIXED))
    assert _rel(g, ref) < 2e-3


@pytest.mark.parametrize("precision", ["f32", "f32acc64"])
def test_fixed_step_fp32_forward_gradient_against_oracle(fq, small, precision):
    # With no step controller the FP32 tracer takes the oracle's steps up to the
    # float rounding of each line's step, so its gradient stays far closer to
    # the oracle's than the RKF45 one does
    B, _, grid = small
    B32 = B.astype(np.float32)
    field = _field(fq, B32, grid)
    m = PLANE16[3] * PLANE16[4]
    wq, wt = _weights(23, m)
    Bd = B32.astype(np.float64)
    Qo = oracle.plane(Bd, grid, *PLANE16, oracle.params(**FIXED))["Q"]
    wq = wq / np.where(np.isfinite(Qo), Qo, 1.0)
    g, _ = _gpu_vjp(fq, field, PLANE16, wq, wt, dtype=torch.float32, precision=precision, **FIXED)
    ref, _ = adj.vjp(Bd, grid, *PLANE16, wq, wt, oracle.params(**FIXED))
    # (measured: 2.9e-5 on the 24^3 cube, both node-grid precisions)
    assert _rel(g, ref) < 5e-4
    assert abs(np.sum(g * Bd)) < 1e-4 * np.linalg.norm(g) * np.linalg.norm(Bd)


@pytest.mark.parametrize("precision,rtol", [("f64", 1e-5), ("f32", 2e-3)])
def test_fixed_step_hyperbolic_closed_form(fq, precision, rtol):
    # B = (x, -y, 1), the closed form of the hyperbolic test above, through the
    # 3/8 rule at 0.2 cells (its footpoints are exact to 1e-7 there)
    grid = synth.ANALYTIC_GRID
    B = synth.analytic_cube("hyperbolic", grid)
    field = _field(fq, B if precision == "f64" else B.astype(np.float32), grid)
    X, Y, Z = _mesh(grid)
    dB = np.stack([X, -Y, 0 * X], -1)
    w = np.random.default_rng(3).uniform(0.5, 1.5, 36)
    g, st = _gpu_vjp(fq, field, PATCH, w, 0 * w, precision=precision, scheme=1, step=0.2, step_min=0.01)
    assert not (st & (oracle.BAD | oracle.MIXED)).any()
    closed = 2.0 * (math.exp(2.0) - math.exp(-2.0))
    np.testing.assert_allclose(np.sum(g * dB), np.sum(w) * closed, rtol=rtol)


def test_fixed_step_checkpoint_interval_and_orthogonality(fq, small):
    B, _, grid = small
    field = _field(fq, B, grid)
    m = PLANE16[3] * PLANE16[4]
    wq, wt = _weights(24, m)
    gs = [_gpu_vjp(fq, field, PLANE16, wq, wt, precision="f64", tape_chunk=k, **FIXED)[0] for k in (1, 7, 32)]
    for g in gs[1:]:
        assert _rel(g, gs[0]) < 1e-12
    assert abs(np.sum(gs[0] * B)) < 1e-11 * np.linalg.norm(gs[0]) * np.linalg.norm(B)


def test_fixed_step_full_size_workload_sampled(fq):
    # the differentiation workload at full size with the fixed-step scheme
    # (step_perp = 3 cells scaled by Eq. step): weights on a seeded sample of 32
    # seeds, against the oracle adjoint traced for those lines and their
    # neighbours
    B, _, grid = synth.adjoint_cubes(seed=2208, n=(128, 128, 64))
    plane = ((0.0, 0.0, 0.0), (127.0 / 256, 0.0, 0.0), (0.0, 127.0 / 256, 0.0), 256, 256)
    n = 256 * 256
    rng = np.random.default_rng(2209)
    sample = np.sort(rng.choice(n, 32, replace=False))
    wq, wt = rng.standard_normal(32), rng.standard_normal(32)
    WQ, WT = np.zeros(n), np.zeros(n)
    WQ[sample], WT[sample] = wq, wt
    ref, _ = adj.vjp_sample(B.astype(np.float64), grid, *plane, sample, wq, wt, oracle.params(scheme=1))
    assert np.linalg.norm(ref) > 0
    field = _field(fq, B, grid)
    g64, _ = _gpu_vjp(fq, field, plane, WQ, WT, precision="f64", scheme=1)
    assert _rel(g64, ref) < 1e-10
    g32, _ = _gpu_vjp(fq, field, plane, WQ, WT, dtype=torch.float32, precision="f32", scheme=1)
    # (measured 1.0e-4 on the benchmark's 64-seed sample)
    assert _rel(g32, ref) < 2e-3


@pytest.mark.parametrize("scheme", [0, 1], ids=["rkf45", "fixed_step"])
def test_gradient_matches_central_differences_of_gpu_maps(fq, small, scheme):
    # The FP64 GPU gradient of the loss against central differences of the
    # GPU's own FP64 maps, each a free re-trace (steps chosen afresh), over the
    # unperturbed map's usable seeds. Tight tolerance / small step, where the
    # frozen step sequence moves the map by much less than the differences
    # resolve (the bounds of the oracle's own finite-difference pins).
    B, Bt, grid = small
    plane = ((0.0, 0.0, 0.0), (23.0 / 8, 0.0, 0.0), (0.0, 23.0 / 8, 0.0), 8, 8)
    kw = dict(precision="f64", tol=1e-8, max_steps=10 ** 6)
    if scheme:
        kw.update(scheme=1, step=0.3, step_min=0.05)
    ft = _field(fq, Bt, grid)
    tgt = {k: v.cpu().numpy() for k, v in fq.qmap_plane(ft, *plane, fq.params(**kw)).items() if v is not None}
    field = _field(fq, B, grid)
    out = fq.qmap_plane(field, *plane, fq.params(tape=1, **kw))
    Q, Tw, st = (out[k].cpu().numpy() for k in ("Q", "Tw", "status"))
    use = (np.isfinite(Q) & np.isfinite(tgt["Q"]) & (Q > 0) & (tgt["Q"] > 0) & np.isfinite(Tw)
           & np.isfinite(tgt["Tw"]) & ((st & (oracle.BAD | oracle.MIXED)) == 0))
    nuse = int(use.sum())
    assert nuse > 40
    r = np.log10(np.where(use, Q, 1.0)) - np.log10(np.where(use, tgt["Q"], 1.0))
    dQ = np.where(use, 2.0 * r / (np.where(use, Q, 1.0) * math.log(10.0) * nuse), 0.0)
    dTw = np.where(use, 0.2 * (Tw - tgt["Tw"]) / nuse, 0.0)
    g = fq.backward(field, torch.from_numpy(dQ).cuda(), torch.from_numpy(dTw).cuda(), dtype=torch.float64)
    field.check()
    g = g.cpu().numpy().ravel()

    def loss(Bx):
        field.update(torch.from_numpy(Bx).cuda())
        o = fq.qmap_plane(field, *plane, fq.params(**kw))
        q, tw = o["Q"].cpu().numpy()[use], o["Tw"].cpu().numpy()[use]
        lq = np.log10(q) - np.log10(tgt["Q"][use])
        return float(np.sum(lq * lq + 0.1 * (tw - tgt["Tw"][use]) ** 2) / nuse)

    flat = np.abs(g)
    cand = np.nonzero(flat > 1e-2 * flat.max())[0]
    pick = np.random.default_rng(31).choice(cand, min(48, len(cand)), replace=False)
    eps = 1e-3 * float(np.sqrt(np.mean(B * B)))
    err = []
    for k in pick:
        Bp = B.copy().ravel()
        Bm = B.copy().ravel()
        Bp[k] += eps
        Bm[k] -= eps
        err.append((loss(Bp.reshape(B.shape)) - loss(Bm.reshape(B.shape))) / (2 * eps) - g[k])
    err = np.abs(np.array(err))
    assert err.max() < 1e-2 * flat.max()
    assert np.median(err / flat[pick]) < 1e-2
