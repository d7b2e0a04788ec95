"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every symbol declared in include/fqsl.h; parameter defaults; and
argument errors that are detected before any CUDA call."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    path = __graft_entry__._builder().build()
    return C.CDLL(path)


def declared_symbols(header="fqsl.h", api="FQSL_API"):
    text = open(os.path.join(ROOT, "include", header)).read()
    return sorted(set(re.findall(api + r"\s+[\w\s\*]*?\b(fqsl_\w+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("fqsl_field_create", "fqsl_qmap_plane", "fqsl_qmap_volume", "fqsl_twist", "fqsl_field_destroy",
              "fqsl_last_error", "fqsl_backward", "fqsl_tape_destroy"):
        assert n in names


def test_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_probe_library_exports_its_symbols():
    # the roofline probes (include/fqsl_probes.h) live in their own library
    import __graft_entry__

    probes = C.CDLL(__graft_entry__._builder().build_probes())
    names = declared_symbols("fqsl_probes.h", "FQSL_PROBE_API")
    assert names == ["fqsl_probe_fma", "fqsl_probe_gather"]
    for name in names:
        assert hasattr(probes, name), name
    # argument errors are refused before any launch
    probes.fqsl_probe_gather.restype = C.c_int
    probes.fqsl_probe_fma.restype = C.c_int
    assert probes.fqsl_probe_gather(None, 8, 8, 8, 0, 1, 1, 1, None, None) == 1
    assert probes.fqsl_probe_gather(C.c_void_p(4096), 2, 8, 8, 0, 1, 1, 1, C.c_void_p(4096), None) == 1
    assert probes.fqsl_probe_gather(C.c_void_p(4096), 8, 8, 8, 7, 1, 1, 1, C.c_void_p(4096), None) == 1
    assert probes.fqsl_probe_fma(0, 0, 1, 1, C.c_void_p(4096), None) == 1


def test_params_defaults():
    import paper_2208_12569_gb300 as fq

    p = fq.params()
    assert p.method == 1 and p.precision == fq.F32
    assert abs(p.tol - 10 ** -3.2) < 1e-15 and p.h0 == 0.5 and p.h_max == 4.0 and p.max_steps == 100000
    assert fq.params(precision="f64").precision == fq.F64
    # the tail of the struct (catches a layout mismatch with the header)
    assert p.sync_dirs == -1 and p.chunk_tiles == 0 and p.blocks_per_sm == 0 and p.refill_lanes == 0
    assert p.eps_way2 == 1e-3 and p.graze == 1e-3
    assert p.tape == 0 and p.tape_chunk == 0 and p.reverse_precision == -1 and p.qperp == 0
    assert p.scheme == 0 and p.step == 3.0 and p.step_min == 0.15


def test_host_argument_errors(lib):
    lib.fqsl_field_create.restype = C.c_int
    lib.fqsl_last_error.restype = C.c_char_p
    h = C.c_void_p()
    o = (C.c_double * 3)(0, 0, 0)
    d = (C.c_double * 3)(1, 1, 1)
    assert lib.fqsl_field_create(None, 0, C.c_longlong(4), C.c_longlong(4), C.c_longlong(4), o, d, 1, None,
                                 C.byref(h)) == 1
    assert b"NULL" in lib.fqsl_last_error()
    fake = C.c_void_p(4096)
    assert lib.fqsl_field_create(fake, 0, C.c_longlong(1), C.c_longlong(4), C.c_longlong(4), o, d, 1, None,
                                 C.byref(h)) == 1
    bad = (C.c_double * 3)(1, 0, 1)
    assert lib.fqsl_field_create(fake, 0, C.c_longlong(4), C.c_longlong(4), C.c_longlong(4), o, bad, 1, None,
                                 C.byref(h)) == 1
    assert lib.fqsl_field_create(fake, 0, C.c_longlong(4), C.c_longlong(4), C.c_longlong(4), o, d, 0, None,
                                 C.byref(h)) == 1
    assert lib.fqsl_field_create(fake, 7, C.c_longlong(4), C.c_longlong(4), C.c_longlong(4), o, d, 1, None,
                                 C.byref(h)) == 1
    # node counts whose product overflows 64 bits (each axis below 2^23) are refused on the host
    big = C.c_longlong(1 << 22)
    assert lib.fqsl_field_create(fake, 0, big, big, big, o, d, 1, None, C.byref(h)) == 1
    assert b"too large" in lib.fqsl_last_error()
    lib.fqsl_qmap_plane.restype = C.c_int
    assert lib.fqsl_qmap_plane(None, o, o, o, C.c_longlong(1), C.c_longlong(1), None, None, None, None) == 1
    # the tape handle's entry points refuse NULL handles on the host
    lib.fqsl_tape_destroy.restype = C.c_int
    lib.fqsl_backward.restype = C.c_int
    lib.fqsl_tape_export.restype = C.c_int
    assert lib.fqsl_tape_destroy(None) == 1
    assert lib.fqsl_backward(None, None, None, None, C.c_void_p(4096), 0, None) == 1
    assert lib.fqsl_tape_export(None, 0, C.c_void_p(4096), C.c_void_p(4096), C.c_void_p(4096), None, None) == 1
    assert b"NULL tape" in lib.fqsl_last_error()


def test_stretched_grid_argument_errors(lib):
    # fqsl_field_create_rect checks its coordinate arrays on the host before
    # touching the device
    lib.fqsl_field_create_rect.restype = C.c_int
    lib.fqsl_last_error.restype = C.c_char_p
    h = C.c_void_p()
    fake = C.c_void_p(4096)
    n = C.c_longlong(4)
    good = (C.c_double * 4)(0.0, 0.5, 1.5, 3.0)
    flat = (C.c_double * 4)(0.0, 0.5, 0.5, 3.0)
    nan = (C.c_double * 4)(0.0, float("nan"), 1.5, 3.0)
    tiny = (C.c_double * 4)(0.0, 1e6, 1e6 + 1e-4, 2e6)  # float keeps about 7 digits of x - x_0

    def create(x, y, z, flags=1):
        return lib.fqsl_field_create_rect(fake, 0, n, n, n, x, y, z, flags, None, C.byref(h))

    assert create(good, None, good) == 1 and b"NULL" in lib.fqsl_last_error()
    assert create(good, flat, good) == 1 and b"increasing" in lib.fqsl_last_error()
    assert create(nan, good, good) == 1 and b"finite" in lib.fqsl_last_error()
    # cells that float cannot tell apart are refused for FP32 records only
    assert create(good, good, tiny, 1) == 1 and b"float" in lib.fqsl_last_error()
    assert create(good, good, good, 0) == 1
    assert lib.fqsl_field_create_rect(None, 0, n, n, n, good, good, good, 1, None, C.byref(h)) == 1


# (field, bad value, phrase of the message): each violates one documented
# range of fqsl_params and is refused before the field handle is read
BAD_PARAMS = [
    ("method", 3, b"method"), ("gradb_way", 0, b"gradb_way"), ("precision", 7, b"precision"),
    ("tol", 0.0, b"tol must be"), ("tol", float("nan"), b"tol must be"), ("tol", float("inf"), b"tol must be"),
    ("h_min", 0.0, b"h_min"), ("h0", 10.0, b"h_min <= h0 <= h_max"), ("h_max", float("inf"), b"h_max"),
    ("max_steps", 0, b"max_steps"), ("max_steps", 3 * 10 ** 9, b"max_steps"), ("rot_thresh", 1.0, b"rot_thresh"),
    ("rot_thresh", -0.1, b"rot_thresh"), ("tol_exp", -1.0, b"tol_exp"), ("graze", 0.0, b"graze"),
    ("graze", 1.0, b"graze"), ("eps_way2", 0.5, b"eps_way2"), ("refill_lanes", 33, b"refill_lanes"),
    ("refill_lanes", -1, b"refill_lanes"), ("sync_dirs", 2, b"sync_dirs"), ("chunk_tiles", 65, b"chunk_tiles"),
    ("blocks_per_sm", 65, b"blocks_per_sm"), ("tape", 2, b"tape must be"), ("tape_chunk", 33, b"tape_chunk"),
    ("reverse_precision", 5, b"reverse_precision"),
]


@pytest.mark.parametrize("name,value,phrase", BAD_PARAMS)
def test_params_out_of_range_are_refused_on_the_host(lib, name, value, phrase):
    import paper_2208_12569_gb300 as fq
    from paper_2208_12569_gb300 import fqsl as fqm

    lib.fqsl_qmap_plane.restype = C.c_int
    lib.fqsl_qmap_volume.restype = C.c_int
    lib.fqsl_twist.restype = C.c_int
    lib.fqsl_last_error.restype = C.c_char_p
    p = fq.params()
    setattr(p, name, value)
    fake = C.c_void_p(4096)  # never read: the parameters are checked first
    o = (C.c_double * 3)(0, 0, 0)
    e = (C.c_double * 3)(1, 0, 0)
    f = (C.c_double * 3)(0, 1, 0)
    out = fqm.Out()
    ll = C.c_longlong
    assert lib.fqsl_qmap_plane(fake, o, e, f, ll(4), ll(4), C.byref(p), C.byref(out), None, None) == 1
    assert phrase in lib.fqsl_last_error()
    assert lib.fqsl_qmap_volume(fake, o, e, ll(2), ll(2), ll(2), C.byref(p), C.byref(out), None, None) == 1
    assert phrase in lib.fqsl_last_error()
    assert lib.fqsl_twist(fake, C.c_void_p(4096), ll(1), C.byref(p), C.byref(out), None) == 1
    assert phrase in lib.fqsl_last_error()


def test_every_entry_point_refuses_null_handles(lib):
    """Each entry point that takes a handle or output array refuses NULL with
    FQSL_ERR_ARG and a message, before any CUDA call."""
    import paper_2208_12569_gb300 as fq
    from paper_2208_12569_gb300 import fqsl as fqm

    lib.fqsl_last_error.restype = C.c_char_p
    p = fq.params()
    out = fqm.Out()
    o = (C.c_double * 3)(0, 0, 0)
    ll = C.c_longlong
    plane = fqm.Plane()
    fake = C.c_void_p(4096)
    calls = {
        "fqsl_field_update": lambda: lib.fqsl_field_update(None, fake, 0, None),
        "fqsl_field_destroy": lambda: lib.fqsl_field_destroy(None),
        "fqsl_field_set_timing": lambda: lib.fqsl_field_set_timing(None, 1),
        "fqsl_field_times": lambda: lib.fqsl_field_times(None, (C.c_float * 3)()),
        "fqsl_field_check": lambda: lib.fqsl_field_check(None, None),
        "fqsl_qmap_volume": lambda: lib.fqsl_qmap_volume(None, o, o, ll(1), ll(1), ll(1), C.byref(p), C.byref(out),
                                                         None, None),
        "fqsl_twist": lambda: lib.fqsl_twist(None, fake, ll(1), C.byref(p), C.byref(out), None),
        "fqsl_qmap_plane_static": lambda: lib.fqsl_qmap_plane_static(None, o, o, o, ll(1), ll(1), C.byref(p),
                                                                     C.byref(out), None),
        "fqsl_batch_create": lambda: lib.fqsl_batch_create(None, C.byref(plane), C.byref(out), 1, C.byref(p),
                                                           C.byref(C.c_void_p())),
        "fqsl_batch_run": lambda: lib.fqsl_batch_run(None, None),
        "fqsl_batch_destroy": lambda: lib.fqsl_batch_destroy(None),
        "fqsl_loss_logq_tw": lambda: lib.fqsl_loss_logq_tw(ll(4), None, fake, fake, fake, None, C.c_double(0.1),
                                                           fake, None, None, None, None),
    }
    for name, call in calls.items():
        getattr(lib, name).restype = C.c_int
        assert call() == 1, name
        assert lib.fqsl_last_error(), name
    # the batch's other arguments
    lib.fqsl_batch_create.restype = C.c_int
    h = C.c_void_p(fake.value)
    assert lib.fqsl_batch_create(C.byref(fake), C.byref(plane), C.byref(out), 1, C.byref(p), None) == 1
    assert lib.fqsl_batch_create(C.byref(fake), C.byref(plane), C.byref(out), 0, C.byref(p), C.byref(h)) == 1
    assert h.value is None  # *out is cleared on refusal
    assert lib.fqsl_batch_create(C.byref(fake), C.byref(plane), C.byref(out), 1, None, C.byref(h)) == 1
    p2 = fq.params(method=2)
    lib.fqsl_batch_create(C.byref(fake), C.byref(plane), C.byref(out), 1, C.byref(p2), C.byref(h))
    assert b"Method I" in lib.fqsl_last_error()
    # the loss: a negative count and a non-finite weight
    lib.fqsl_loss_logq_tw.restype = C.c_int
    assert lib.fqsl_loss_logq_tw(ll(-1), fake, fake, fake, fake, None, C.c_double(0.1), fake, None, None, None,
                                 None) == 1
    assert lib.fqsl_loss_logq_tw(ll(4), fake, fake, fake, fake, None, C.c_double(float("nan")), fake, None, None,
                                 None, None) == 1
    assert b"w_tw" in lib.fqsl_last_error()
    # the tape export: a negative cap and NULL outputs
    lib.fqsl_tape_export.restype = C.c_int
    assert lib.fqsl_tape_export(fake, -1, fake, fake, fake, fake, None) == 1
    assert lib.fqsl_tape_export(fake, 4, fake, fake, fake, None, None) == 1
    assert b"NULL output" in lib.fqsl_last_error()
