"""Out-of-memory paths, made on demand with the library's allocation cap
(fqsl_debug_alloc_cap): no GPU is exhausted, faulted or hung. Each failing
call returns FQSL_ERR_OOM (status 3) before any launch that would need the
memory, leaves nothing half-built behind, and the same call succeeds once the
cap is lifted."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

OOM = 3


@pytest.fixture(scope="module")
def fq():
    import paper_2208_12569_gb300 as fq

    return fq


@pytest.fixture(autouse=True)
def _no_cap(fq):
    yield
    fq.debug_alloc_cap(0)


def _cube():
    grid = synth.Grid((40, 36, 24), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    B = synth.monopole_cube(grid, synth.random_charges(np.random.default_rng(5), 6, ((0.0, 39.0), (0.0, 35.0))))
    return torch.from_numpy(np.ascontiguousarray(B, dtype=np.float32)).cuda(), grid


def test_field_records_out_of_memory(fq):
    B, grid = _cube()
    nodes = 40 * 36 * 24
    fq.debug_alloc_cap(nodes * 32 - 1)  # the FP32 records do not fit
    with pytest.raises(fq.FqslError) as e:
        fq.Field(B, grid.origin, grid.spacing, pack=("f32",))
    assert e.value.status == OOM and "out of memory" in str(e.value)
    fq.debug_alloc_cap(0)
    f = fq.Field(B, grid.origin, grid.spacing, pack=("f32",))
    out = fq.qmap_plane(f, (0, 0, 0), (39.0 / 32, 0, 0), (0, 35.0 / 32, 0), 32, 32, fq.params(precision="f32"))
    assert int(torch.isfinite(out["Q"]).sum()) > 500
    f.close()


def test_map_scratch_and_tape_out_of_memory(fq):
    B, grid = _cube()
    f = fq.Field(B, grid.origin, grid.spacing, pack=("f64",))
    plane = ((0, 0, 0), (39.0 / 32, 0, 0), (0, 35.0 / 32, 0), 32, 32)
    p = fq.params(precision="f64")
    ref = fq.qmap_plane(f, *plane, p)
    big = ((0, 0, 0), (39.0 / 256, 0, 0), (0, 35.0 / 256, 0), 256, 256)
    fq.debug_alloc_cap(1 << 20)  # the larger map's scratch does not fit in 1 MiB
    with pytest.raises(fq.FqslError) as e:
        fq.qmap_plane(f, *big, p)
    assert e.value.status == OOM
    # a taped map: its tape buffer does not fit either
    with pytest.raises(fq.FqslError) as e:
        fq.qmap_plane(f, *plane, fq.params(precision="f64", tape=1))
    assert e.value.status == OOM
    fq.debug_alloc_cap(0)
    again = fq.qmap_plane(f, *plane, p)
    for k in ("Q", "Tw", "r1", "r2", "status", "steps"):
        assert torch.equal(torch.nan_to_num(again[k]), torch.nan_to_num(ref[k])), k
    out = fq.qmap_plane(f, *plane, fq.params(precision="f64", tape=1))
    dB = fq.backward(f, dQ=torch.ones(32 * 32, dtype=torch.float64, device="cuda"), dtype=torch.float64)
    f.check()
    assert torch.isfinite(dB).all() and float(dB.abs().sum()) > 0
    assert torch.equal(torch.nan_to_num(out["Q"]), torch.nan_to_num(ref["Q"]))
    f.close()
