"""Batches (one set of launches over many cubes and planes of uneven sizes):
every entry equals the single-plane entry point's result bit for bit, in both
precisions and with both integration schemes, including interior planes that
rotate S0; a captured CUDA graph replays to the same results."""
import numpy as np
import pytest

import synth
from parity import assert_bitwise, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_12569_gb300 as fq

    rng = np.random.default_rng(77)
    shapes = [(40, 36, 24), (64, 48, 32), (33, 29, 17)]
    fields, planes = [], []
    for k, n in enumerate(shapes):
        grid = synth.Grid(n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
        ch = synth.random_charges(rng, 6 + 3 * k, ((0.0, n[0] - 1.0), (0.0, n[1] - 1.0)), depth=(3.0, 9.0))
        B = synth.monopole_cube(grid, ch, dtype=np.float32)
        fields.append(fq.Field(torch.from_numpy(B).cuda(), grid.origin, grid.spacing))
        nu, nv = 37 + 11 * k, 23 + 5 * k
        # a face plane and an interior vertical plane (S0 rotation) per cube
        planes.append(dict(origin=(0.0, 0.0, 0.0), u=((n[0] - 1.0) / nu, 0.0, 0.0), v=(0.0, (n[1] - 1.0) / nv, 0.0),
                           nu=nu, nv=nv))
        planes.append(dict(origin=(0.0, (n[1] - 1.0) * 0.37, 0.0), u=((n[0] - 1.0) / nu, 0.0, 0.0),
                           v=(0.0, 0.0, (n[2] - 1.0) / nv), nu=nu, nv=nv))
    fields = [f for f in fields for _ in range(2)]
    return fq, fields, planes


@pytest.mark.parametrize("scheme", [0, 1], ids=["rkf45", "fixed_step"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batch_equals_single_entries(setup, precision, scheme):
    # (scheme 1: the fixed-step 3/8 rule with Eq. step's per-line step, Sec. 2.3)
    fq, fields, planes = setup
    p = fq.params(precision=precision, scheme=scheme)
    batch = fq.Batch(fields, planes, p)
    outs = [to_np(o) for o in batch.run()]
    torch.cuda.synchronize()
    rotated = 0
    for fld, pl, got in zip(fields, planes, outs):
        ref = to_np(fq.qmap_plane(fld, pl["origin"], pl["u"], pl["v"], pl["nu"], pl["nv"], p))
        fld.check()
        assert_bitwise(got, ref)
        rotated += int((ref["status"] & fq.LINE_ROTATED).astype(bool).sum())
    assert rotated > 0
    batch.close()


def test_batch_graph_replay(setup):
    fq, fields, planes = setup
    p = fq.params(precision="f32")
    batch = fq.Batch(fields, planes, p)
    ref = [to_np(o) for o in batch.run()]
    g = batch.graph()
    for o in batch.outs:
        for t in o.values():
            if t is not None:
                t.fill_(3)
    g.replay()
    torch.cuda.synchronize()
    for o, r in zip(batch.outs, ref):
        assert_bitwise(to_np(o), r)
    batch.close()
