"""The two largest configurations at full size, in the launch configuration the
benchmark times, against the oracle on seeded samples of seeds that it
recomputes one by one (each Method I seed with its four lattice neighbours):

- the batch of 48 uneven monopole cubes (64^3 to 384^2x192 nodes, 512x256
  seeds each, 6.29 M lines) traced in one set of launches: FP64 bit-identical
  and FP32 error stated on sampled entries;
- the 1024x1024x512 monopole cube: the 512x512x256 cell-centred seed volume
  (FP32 and FP64) and the 4096x4096 z=0 map (FP32)."""
import numpy as np
import pytest

import oracle
import synth
from parity import assert_bitwise, assert_fp64_parity, q_rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2208_12569_gb300 as m

    return m


def _take(out, idx):
    """Host copies of the sampled entries of a map's outputs."""
    it = torch.from_numpy(idx).to(out["Q"].device)
    return {k: t.index_select(0, it).cpu().numpy() for k, t in out.items() if t is not None}


def _check_fp32(g, r):
    assert np.mean(g["face2"] == r["face2"]) > 0.98
    rel = q_rel(g, r)
    assert np.median(rel[np.isfinite(rel)]) < 1e-3


def test_batch48_full_size_sampled(fq):
    dev = torch.device("cuda", 0)
    specs = synth.batch_specs(seed=2208)
    cubes = [synth.monopole_cube(sp["grid"], sp["charges"], dtype=np.float32, device=dev) for sp in specs]
    fields = [fq.Field(B, sp["grid"].origin, sp["grid"].spacing, pack=("f32", "f64")) for B, sp in zip(cubes, specs)]
    planes = [sp["plane"] for sp in specs]
    rng = np.random.default_rng(2208)
    # six entries: the largest cube size present and five seeded others
    largest = max(range(len(specs)), key=lambda k: int(np.prod(specs[k]["grid"].n)))
    pick = [largest] + [int(k) for k in rng.choice([k for k in range(len(specs)) if k != largest], 5, replace=False)]
    samples = {k: np.sort(rng.choice(planes[k]["nu"] * planes[k]["nv"], 300, replace=False)) for k in pick}
    got = {}
    for prec in ("f64", "f32"):
        batch = fq.Batch(fields, planes, fq.params(precision=prec))
        outs = batch.run()
        torch.cuda.synchronize()
        got[prec] = {k: _take(outs[k], samples[k]) for k in pick}
        batch.close()
    for f in fields:
        f.check()
    for k in pick:
        sp, pl = specs[k], planes[k]
        r = oracle.plane(cubes[k].cpu().numpy().astype(np.float64), sp["grid"], pl["origin"], pl["u"], pl["v"],
                         pl["nu"], pl["nv"], oracle.params(), sample=samples[k])
        assert_fp64_parity(got["f64"][k], r)
        assert_bitwise(got["f64"][k], r)
        _check_fp32(got["f32"][k], r)
    for f in fields:
        f.close()


def test_large_volume_full_size_sampled(fq):
    dev = torch.device("cuda", 0)
    n = (1024, 1024, 512)
    Bd, grid, _ = synth.large_monopole(n=n, device=dev)
    vol = (512, 512, 256)
    step = tuple((n[a] - 1.0) / vol[a] for a in range(3))
    nplane = 4096
    u, v = ((n[0] - 1.0) / nplane, 0.0, 0.0), (0.0, (n[1] - 1.0) / nplane, 0.0)
    rng = np.random.default_rng(2208)
    sv = np.sort(rng.choice(vol[0] * vol[1] * vol[2], 1500, replace=False))
    sp = np.sort(rng.choice(nplane * nplane, 1000, replace=False))
    field = fq.Field(Bd, grid.origin, grid.spacing, pack=("f32",))
    g32v = _take(fq.qmap_volume(field, (0.0, 0.0, 0.0), step, *vol, fq.params(precision="f32")), sv)
    g32p = _take(fq.qmap_plane(field, (0.0, 0.0, 0.0), u, v, nplane, nplane, fq.params(precision="f32")), sp)
    field.check()
    field.close()
    torch.cuda.empty_cache()
    field = fq.Field(Bd, grid.origin, grid.spacing, pack=("f64",))
    g64v = _take(fq.qmap_volume(field, (0.0, 0.0, 0.0), step, *vol, fq.params(precision="f64")), sv)
    field.check()
    field.close()
    B64 = Bd.cpu().numpy().astype(np.float64)
    del Bd
    torch.cuda.empty_cache()
    J = oracle.curl(B64, grid)
    rv = oracle.qmap(B64, grid, (0.0, 0.0, 0.0), (step[0], 0, 0), (0, step[1], 0), (0, 0, step[2]), vol,
                     oracle.params(), sample=sv, J=J)
    assert_fp64_parity(g64v, rv)
    assert_bitwise(g64v, rv)
    _check_fp32(g32v, rv)
    rp = oracle.plane(B64, grid, (0.0, 0.0, 0.0), u, v, nplane, nplane, oracle.params(), sample=sp, J=J)
    _check_fp32(g32p, rp)
