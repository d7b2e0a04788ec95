"""FP64 CPU oracle for the FastQSL method -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product library (the CUDA path)
never calls it and shares no code with it. The arithmetic lives in
``fqsl_oracle.c`` (plain C, compiled with floating-point contraction off so the
same results come out on x86-64 and aarch64); this module only builds it and
marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fqsl_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# line status bits (reading R11 in fqsl_oracle.c)
MAXSTEPS, NULL_B, STALL, MIXED, OUTSIDE, ROTATED, CHORD = 1, 2, 4, 8, 16, 32, 64
BAD = MAXSTEPS | NULL_B | OUTSIDE


def build(force: bool = False) -> str:
    """Compile fqsl_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("method", C.c_int), ("way", C.c_int), ("tol", C.c_double), ("h0", C.c_double),
                ("hmin", C.c_double), ("hmax", C.c_double), ("max_steps", C.c_longlong),
                ("rot_thresh", C.c_double), ("tol_exp", C.c_double), ("graze", C.c_double),
                ("eps2", C.c_double), ("qperp", C.c_int), ("scheme", C.c_int), ("step", C.c_double),
                ("step_min", C.c_double)]


def params(method=1, way=1, tol=10 ** -3.2, h0=0.5, hmin=1e-6, hmax=4.0, max_steps=100000,
           rot_thresh=0.05, tol_exp=1.5, graze=1e-3, eps2=1e-3, qperp=0, scheme=0, step=3.0,
           step_min=0.15) -> Params:
    """Oracle parameters (readings R2, R5, R9, R10, R17, R18 of fqsl_oracle.c);
    qperp = 1 gives Q_perp (Method II); scheme = 1 the fixed-step 3/8-rule RK4
    with step_perp = step and Eq. step's floor step_min."""
    return Params(method, way, tol, h0, hmin, hmax, max_steps, rot_thresh, tol_exp, graze, eps2, qperp, scheme,
                  step, step_min)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            for name in ("oracle_curl", "oracle_gradb", "oracle_interp", "oracle_qmap", "oracle_twist",
                         "oracle_trace", "oracle_max_threads", "oracle_curl_rect", "oracle_qmap_rect",
                         "oracle_twist_rect", "oracle_interp_rect", "oracle_cell_rect", "oracle_gradb_rect",
                         "oracle_lattice_log_rect"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def is_rect(grid) -> bool:
    """A stretched grid (node coordinate arrays, reading R16) rather than a
    uniform one."""
    return hasattr(grid, "coords")


def _coords(grid):
    return np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.float64) for c in grid.coords]))


def _grid_args(grid):
    if is_rect(grid):
        raise ValueError("this oracle function takes a uniform grid")
    n = np.array(grid.n, dtype=np.int64)
    o = np.array(grid.origin, dtype=np.float64)
    d = np.array(grid.spacing, dtype=np.float64)
    return n, o, d


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def curl(B, grid):
    """curl B at the nodes (same layout as B, float64)."""
    B = _f64(B)
    J = np.empty_like(B)
    if is_rect(grid):
        n = np.array(grid.n, dtype=np.int64)
        rc = lib().oracle_curl_rect(_p(B), _p(n), _p(_coords(grid)), _p(J))
        if rc:
            raise ValueError("oracle_curl_rect: bad grid")
        return J
    n, o, d = _grid_args(grid)
    rc = lib().oracle_curl(_p(B), _p(n), _p(d), _p(J))
    if rc:
        raise ValueError("oracle_curl: bad grid")
    return J


def gradb(B, grid):
    """d(B_b/|B|)/dx_a at the nodes, shape (nz, ny, nx, 9), index a*3+b."""
    B = _f64(B)
    G = np.empty(B.shape[:3] + (9,), dtype=np.float64)
    if is_rect(grid):
        n = np.array(grid.n, dtype=np.int64)
        if lib().oracle_gradb_rect(_p(B), _p(n), _p(_coords(grid)), _p(G)):
            raise ValueError("oracle_gradb_rect: bad grid")
        return G
    n, o, d = _grid_args(grid)
    rc = lib().oracle_gradb(_p(B), _p(n), _p(d), _p(G))
    if rc:
        raise ValueError("oracle_gradb: bad grid")
    return G


def interp(arr, n, xi):
    """Trilinear interpolation of node array ``arr`` (nz,ny,nx,nc) at index
    coordinates ``xi`` (m, 3)."""
    arr = _f64(arr)
    nc = arr.shape[-1]
    xi = _f64(np.atleast_2d(xi))
    out = np.empty((xi.shape[0], nc))
    nn = np.array(n, dtype=np.int64)
    lib().oracle_interp(_p(arr), C.c_int(nc), _p(nn), _p(xi), C.c_longlong(xi.shape[0]), _p(out))
    return out


def interp_rect(arr, grid, r):
    """Trilinear interpolation (Eqs. interp, w0, w1) of node array ``arr``
    (nz,ny,nx,nc) on the stretched grid at physical points ``r`` (m, 3)."""
    arr = _f64(arr)
    nc = arr.shape[-1]
    r = _f64(np.atleast_2d(r))
    out = np.empty((r.shape[0], nc))
    n = np.array(grid.n, dtype=np.int64)
    rc = lib().oracle_interp_rect(_p(arr), C.c_int(nc), _p(n), _p(_coords(grid)), _p(r), C.c_longlong(r.shape[0]),
                                  _p(out))
    if rc:
        raise ValueError("oracle_interp_rect: bad grid")
    return out


def cell_rect(X, x):
    """Cell index of each coordinate x on an axis with node coordinates X."""
    X = _f64(np.asarray(X))
    x = _f64(np.atleast_1d(x))
    out = np.empty(len(x), np.int64)
    if lib().oracle_cell_rect(_p(X), C.c_longlong(len(X)), _p(x), C.c_longlong(len(x)), _p(out)):
        raise ValueError("oracle_cell_rect: bad axis")
    return out


def _prep_field(B, grid, J, G, p):
    B = _f64(B)
    if J is None:
        J = curl(B, grid)
    J = _f64(J)
    if p.method == 2 and p.way == 1 and G is None:
        G = gradb(B, grid)
    G = _f64(G)
    return B, J, G


def qmap(B, grid, origin, a1, a2, a3=(0.0, 0.0, 0.0), counts=(1, 1, 1), p: Params | None = None,
         sample=None, J=None, G=None):
    """Q, Tw, length, footpoints, faces, status and trial-step counts on the
    cell-centred lattice origin + (i+1/2) a1 + (j+1/2) a2 + (k+1/2) a3.

    counts = (n1, n2, n3). ``sample`` = linear lattice indices i + n1 (j + n2 k)
    to compute (default: all, in that order)."""
    p = p or params()
    B, J, G = _prep_field(B, grid, J, G, p)
    lo = np.array(origin, dtype=np.float64)
    A1, A2, A3 = (np.array(v, dtype=np.float64) for v in (a1, a2, a3))
    ln = np.array(counts, dtype=np.int64)
    if sample is not None:
        sample = np.ascontiguousarray(sample, dtype=np.int64)
        m = len(sample)
    else:
        m = int(np.prod(counts))
    out = dict(Q=np.empty(m), Tw=np.empty(m), length=np.empty(m), r1=np.empty((m, 3)),
               r2=np.empty((m, 3)), face1=np.empty(m, np.int32), face2=np.empty(m, np.int32),
               status=np.empty(m, np.int32), steps=np.empty(m, np.int64))
    outs = (_p(out["Q"]), _p(out["Tw"]), _p(out["length"]), _p(out["r1"]), _p(out["r2"]), _p(out["face1"]),
            _p(out["face2"]), _p(out["status"]), _p(out["steps"]))
    if is_rect(grid):
        n = np.array(grid.n, dtype=np.int64)
        rc = lib().oracle_qmap_rect(_p(B), _p(J), _p(G), _p(n), _p(_coords(grid)), _p(lo), _p(A1), _p(A2), _p(A3),
                                    _p(ln), C.byref(p), _p(sample), C.c_longlong(m if sample is not None else 0),
                                    *outs)
    else:
        n, o, d = _grid_args(grid)
        rc = lib().oracle_qmap(_p(B), _p(J), _p(G), _p(n), _p(o), _p(d), _p(lo), _p(A1), _p(A2), _p(A3),
                               _p(ln), C.byref(p), _p(sample), C.c_longlong(m if sample is not None else 0), *outs)
    if rc:
        raise ValueError("oracle_qmap: argument error %d" % rc)
    return out


def plane(B, grid, origin, u, v, nu, nv, p: Params | None = None, sample=None, J=None, G=None):
    """Q map on the plane lattice origin + (i+1/2) u + (j+1/2) v."""
    return qmap(B, grid, origin, u, v, (0.0, 0.0, 0.0), (nu, nv, 1), p, sample, J, G)


def twist(B, grid, seeds, p: Params | None = None, J=None):
    """Tw, length and footpoints for explicit physical seeds (m, 3)."""
    p = p or params()
    B = _f64(B)
    J = _f64(curl(B, grid) if J is None else J)
    seeds = _f64(np.atleast_2d(seeds))
    m = seeds.shape[0]
    out = dict(Tw=np.empty(m), length=np.empty(m), r1=np.empty((m, 3)), r2=np.empty((m, 3)),
               face1=np.empty(m, np.int32), face2=np.empty(m, np.int32), status=np.empty(m, np.int32),
               steps=np.empty(m, np.int64))
    outs = (_p(out["Tw"]), _p(out["length"]), _p(out["r1"]), _p(out["r2"]), _p(out["face1"]), _p(out["face2"]),
            _p(out["status"]), _p(out["steps"]))
    if is_rect(grid):
        n = np.array(grid.n, dtype=np.int64)
        rc = lib().oracle_twist_rect(_p(B), _p(J), _p(n), _p(_coords(grid)), _p(seeds), C.c_longlong(m),
                                     C.byref(p), *outs)
    else:
        n, o, d = _grid_args(grid)
        rc = lib().oracle_twist(_p(B), _p(J), _p(n), _p(o), _p(d), _p(seeds), C.c_longlong(m), C.byref(p), *outs)
    if rc:
        raise ValueError("oracle_twist: argument error %d" % rc)
    return out


def trace(B, grid, seeds, tol, p: Params | None = None, U0=None, V0=None, J=None, G=None):
    """Raw line tracing: end states (m, 2, 11) = [xi(3), length, Tw, U(3), V(3)]
    for the backward (0) and forward (1) ends, faces (m, 2), B at the ends
    (m, 2, 3), status, steps."""
    p = p or params()
    B, J, G = _prep_field(B, grid, J, G, p if U0 is not None else params(method=1))
    n, o, d = _grid_args(grid)
    seeds = _f64(np.atleast_2d(seeds))
    m = seeds.shape[0]
    tol = _f64(np.broadcast_to(np.asarray(tol, dtype=np.float64), (m,)))
    U0 = _f64(None if U0 is None else np.atleast_2d(U0))
    V0 = _f64(None if V0 is None else np.atleast_2d(V0))
    if U0 is not None and p.way == 1 and G is None:
        G = gradb(B, grid)
    ends = np.empty((m, 2, 11))
    faces = np.empty((m, 2), np.int32)
    Bend = np.empty((m, 2, 3))
    st = np.empty(m, np.int32)
    steps = np.empty(m, np.int64)
    rc = lib().oracle_trace(_p(B), _p(J), _p(G), _p(n), _p(o), _p(d), _p(seeds), C.c_longlong(m), _p(tol),
                            _p(U0), _p(V0), C.byref(p), _p(ends), _p(faces), _p(Bend), _p(st), _p(steps))
    if rc:
        raise ValueError("oracle_trace: argument error %d" % rc)
    return dict(ends=ends, faces=faces, Bend=Bend, status=st, steps=steps)


def physical(grid, xi):
    """Index coordinates -> physical coordinates."""
    return np.asarray(grid.origin) + np.asarray(grid.spacing) * np.asarray(xi)
