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


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fqsl.h")).read()
    return sorted(set(re.findall(r"FQSL_API\s+[\w\s\*]*?\b(fqsl_\w+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("fqsl_field_create", "fqsl_qmap_plane", "fqsl_qmap_volume", "fqsl_twist", "fqsl_field_destroy",
              "fqsl_last_error"):
        assert n in names


def test_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_params_defaults():
    import paper_2208_12569_gb300 as fq

    p = fq.params()
    assert p.method == 1 and p.precision == fq.F32
    assert abs(p.tol - 10 ** -3.2) < 1e-15 and p.h0 == 0.5 and p.h_max == 4.0 and p.max_steps == 100000
    assert fq.params(precision="f64").precision == fq.F64
    # the tail of the struct (catches a layout mismatch with the header)
    assert p.sync_dirs == -1 and p.chunk_tiles == 0 and p.blocks_per_sm == 0 and p.refill_lanes == 0
    assert p.eps_way2 == 1e-3 and p.graze == 1e-3


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
    lib.fqsl_qmap_plane.restype = C.c_int
    assert lib.fqsl_qmap_plane(None, o, o, o, C.c_longlong(1), C.c_longlong(1), None, None, None) == 1
