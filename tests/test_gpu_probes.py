"""The roofline probes of libfqsl_probes.so (include/fqsl_probes.h) on the
GPU: they run through the C ABI, and their ceilings are ordered as the access
patterns and pipes imply (neighbouring lanes' gathers coalesce, random ones do
not; GB300's FP64 rate is a small fraction of its FP32 rate)."""
import ctypes as C

import numpy as np
import pytest

import bench

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def test_ceilings_are_ordered(dev):
    c = bench.measure_ceilings(dev, cube=(96, 96, 48), target_ms=1.0)
    assert c["gather_walk_TBs"] > 2.0 * c["gather_random_TBs"] > 0.0
    assert c["gather_tile_TBs"] > 2.0 * c["gather_random_TBs"]
    assert c["fma_f32_TFLOPs"] > 10.0 * c["fma_f64_TFLOPs"] > 0.0


def test_gather_probe_interpolates_the_records(dev):
    # every record equal to (1, 2, 3, 4, 5, 6, 0, 0): each trilinear gather
    # returns 21 (the weights sum to one), so a lane's sum is 21 x gathers
    import __graft_entry__

    lib = C.CDLL(__graft_entry__._builder().build_probes())
    lib.fqsl_probe_gather.restype = C.c_int
    n = (16, 12, 8)
    rec = torch.tensor([1, 2, 3, 4, 5, 6, 0, 0], dtype=torch.float32, device=dev).repeat(n[0] * n[1] * n[2])
    sms, bps, gathers = 4, 2, 50
    for pattern in (0, 1, 2):
        sink = torch.zeros(sms * bps * 128, dtype=torch.float32, device=dev)
        rc = lib.fqsl_probe_gather(C.c_void_p(rec.data_ptr()), *n, pattern, gathers, sms, bps,
                                   C.c_void_p(sink.data_ptr()), None)
        assert rc == 0
        torch.cuda.synchronize()
        np.testing.assert_allclose(sink.cpu().numpy(), 21.0 * gathers, rtol=1e-5)
