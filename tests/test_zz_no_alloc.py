"""The allocation-free plane map (fqsl_qmap_plane_static) against the ordinary
one (fqsl_qmap_plane), through the C ABI.

fqsl_qmap_plane_static is for callers that cannot allocate device memory (an
application whose device memory belongs to its own fixed arena, or a loop that
cannot afford the synchronisation of growing scratch): it keeps its scratch in
a static device array of the library. It must give exactly the outputs of the
ordinary entry point -- the same kernels run -- on repeated calls, since the
shared array keeps the previous call's contents. This file is collected last
so that a run stopping at the first failure has run every other test first.
"""
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

    grid = synth.Grid((64, 56, 32), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    ch = synth.random_charges(np.random.default_rng(2208), 10, ((0.0, 63.0), (0.0, 55.0)), depth=(4.0, 12.0))
    B = synth.monopole_cube(grid, ch, dtype=np.float32)
    field = fq.Field(torch.from_numpy(B).cuda(), grid.origin, grid.spacing)
    return fq, field


# (origin, u, v, nu, nv): the z=0 face plane at the size limit, and an interior
# xz plane whose near-tangent seeds use the rotated-S0 buffers
PLANES = [((0.0, 0.0, 0.0), (63.0 / 256, 0.0, 0.0), (0.0, 55.0 / 256, 0.0), 256, 256),
          ((0.0, 10.3, 0.0), (63.0 / 180, 0.0, 0.0), (0.0, 0.0, 31.0 / 90), 180, 90)]


@pytest.mark.parametrize("plane", PLANES, ids=["face_plane_max_size", "interior_plane_rotated"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_static_entry_point_matches_allocating_one(setup, plane, precision):
    fq, field = setup
    p = fq.params(precision=precision)
    ref = to_np(fq.qmap_plane(field, *plane, p))
    field.check()
    if plane[1][1] == 10.3:
        assert int((ref["status"] & fq.LINE_ROTATED).astype(bool).sum()) > 50
    n = plane[3] * plane[4]
    out = fq.alloc_out(n)
    for _ in range(2):  # two calls in a row reuse the same static scratch
        for t in out.values():
            t.fill_(7)
        got = to_np(fq.qmap_plane_static(field, *plane, p, out=out))
        field.check()
        assert_bitwise(got, ref)


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("case", ["rkf45", "fixed_step", "stretched"])
def test_static_calls_allocate_no_device_memory(setup, case):
    """After a first call (which may load the library's static array), further
    calls leave the device's free memory unchanged: nothing is allocated. The
    fixed-step scheme and a stretched grid take the same path and give the
    ordinary entry point's outputs bit for bit."""
    fq, field = setup
    plane = PLANES[1]
    p = fq.params(precision="f64", scheme=1 if case == "fixed_step" else 0)
    if case == "stretched":
        grid = synth.stretched_grid((64, 56, 32), (0.0, 0.0, 0.0), (63.0, 55.0, 31.0), ratios=(1.03, 1.03, 1.04))
        ch = synth.random_charges(np.random.default_rng(2208), 10, ((0.0, 63.0), (0.0, 55.0)), depth=(4.0, 12.0))
        B = synth.monopole_cube(grid, ch, dtype=np.float32)
        field = fq.Field(torch.from_numpy(B).cuda(), coords=grid.coords)
    ref = to_np(fq.qmap_plane(field, *plane, p))
    field.check()
    n = plane[3] * plane[4]
    out = fq.alloc_out(n)
    fq.qmap_plane_static(field, *plane, p, out=out)  # may load the static array
    field.check()
    free0 = _free_bytes()
    for _ in range(3):
        for t in out.values():
            t.fill_(7)
        fq.qmap_plane_static(field, *plane, p, out=out)
    free1 = _free_bytes()
    field.check()
    assert free1 == free0
    assert_bitwise(to_np(out), ref)


def test_static_entry_point_is_timed(setup):
    # with timing enabled, the static call records its own kernel times
    fq, field = setup
    plane = PLANES[1]
    p = fq.params(precision="f32")
    field.set_timing(True)
    try:
        fq.qmap_plane_static(field, *plane, p, out=fq.alloc_out(plane[3] * plane[4]))
        ms = field.times()
        assert ms[0] > 0.0 and ms[1] > 0.0 and ms[2] > 0.0  # tracer, rotated extra lines, assembly
    finally:
        field.set_timing(False)


def test_static_entry_point_rejects_oversize(setup):
    fq, field = setup
    n = fq.STATIC_MAX_SEEDS + 1
    with pytest.raises(fq.FqslError) as ei:
        fq.qmap_plane_static(field, (0.0, 0.0, 0.0), (0.1, 0.0, 0.0), (0.0, 0.1, 0.0), n, 1)
    assert ei.value.status == 1 and "FQSL_STATIC_MAX_SEEDS" in str(ei.value)
    # a product that would overflow 64 bits (2^32 x 2^32) is refused before any launch
    with pytest.raises(fq.FqslError) as ei:
        fq.qmap_plane_static(field, (0.0, 0.0, 0.0), (0.1, 0.0, 0.0), (0.0, 0.1, 0.0), 1 << 32, 1 << 32,
                             out=fq.alloc_out(1))
    assert ei.value.status == 1 and "FQSL_STATIC_MAX_SEEDS" in str(ei.value)
