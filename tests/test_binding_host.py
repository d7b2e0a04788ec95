"""Host-side logic of the Python binding (paper_2208_12569_gb300/fqsl.py) that
needs no GPU: keyword parameters and their names, the checks on tensors that
are refused before any library call, the tape bookkeeping, and the error type
that carries the library's status."""
import types

import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fq():
    import paper_2208_12569_gb300 as m

    return m


def test_params_keywords(fq):
    p = fq.params(precision="f32acc64", reverse_precision="f64", tol=1e-4, scheme=1, step=2.5, qperp=1, method=2)
    assert p.precision == fq.F32_ACC64 and p.reverse_precision == fq.F64
    assert p.tol == 1e-4 and p.scheme == 1 and p.step == 2.5 and p.qperp == 1 and p.method == 2
    assert fq.params(precision=1).precision == fq.F64
    with pytest.raises(KeyError):
        fq.params(tolerance=1e-3)
    with pytest.raises(KeyError):
        fq.params(precision="bf16")


class _OnDevice(torch.Tensor):
    """A CPU tensor that reports itself as a CUDA one: it passes the binding's
    device check, so the checks after it are reached without a GPU."""

    @property
    def is_cuda(self):
        return True


def _cube(last=3, dtype=torch.float32):
    return torch.zeros((4, 4, 4, last), dtype=dtype).as_subclass(_OnDevice)


def test_field_refuses_bad_tensors_before_the_library(fq):
    with pytest.raises(ValueError, match="CUDA tensor"):
        fq.Field(torch.zeros((4, 4, 4, 3)), (0, 0, 0), (1, 1, 1))
    with pytest.raises(ValueError, match=r"\(nz, ny, nx, 3\)"):
        fq.Field(_cube(last=2), (0, 0, 0), (1, 1, 1))
    with pytest.raises(ValueError, match="float32 or float64"):
        fq.Field(_cube(dtype=torch.float16), (0, 0, 0), (1, 1, 1))


def test_field_grid_arguments_are_exclusive(fq):
    with pytest.raises(ValueError, match="either origin and spacing"):
        fq.Field(_cube(), (0, 0, 0), (1, 1, 1), coords=([0, 1, 2, 3],) * 3)
    with pytest.raises(ValueError, match="either origin and spacing"):
        fq.Field(_cube())


def test_tape_bookkeeping(fq):
    field = types.SimpleNamespace()
    with pytest.raises(RuntimeError, match="no taped map"):
        fq.fqsl._tape_of(field, None)
    # an untaped call takes no tape and leaves the field's record alone
    assert fq.fqsl._tape_arg(field, fq.params(), None) == (None, None)
    assert not hasattr(field, "last_tape")


def test_loss_refuses_non_double_inputs(fq):
    q = torch.ones(4, dtype=torch.float32)
    d = torch.ones(4, dtype=torch.float64)
    with pytest.raises(ValueError, match="float64"):
        fq.loss_logq_tw(q, d, d, d, out=dict(sums=d, loss=d, dQ=d, dTw=d))


def test_error_carries_status(fq):
    e = fq.FqslError(3, "scratch allocation: out of memory")
    assert e.status == 3 and "status 3" in str(e) and isinstance(e, RuntimeError)


def test_version_and_exports(fq):
    assert fq.version().startswith("fqsl ")
    for name in ("Field", "Tape", "Batch", "QTwPlane", "qmap_plane", "qmap_plane_static", "qmap_volume", "twist",
                 "backward", "tape_export", "loss_logq_tw", "debug_alloc_cap", "params", "alloc_out"):
        assert hasattr(fq, name), name
