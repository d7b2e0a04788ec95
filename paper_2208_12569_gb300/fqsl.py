"""Thin Python binding of libfqsl.so (include/fqsl.h).

Argument marshalling only: torch supplies device memory and the current CUDA
stream; every step of the computation runs in the library's CUDA kernels. If
the library is missing this module raises at import time -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfqsl.so")

F32, F64, F32_ACC64 = 0, 1, 2
PACK_F32, PACK_F64, PACK_GRADB = 1, 2, 4
LINE_MAXSTEPS, LINE_NULL_B, LINE_STALL, LINE_MIXED, LINE_OUTSIDE, LINE_ROTATED, LINE_CHORD = 1, 2, 4, 8, 16, 32, 64
LINE_BAD = LINE_MAXSTEPS | LINE_NULL_B | LINE_OUTSIDE
EXPORTS = ("fqsl_params_default", "fqsl_version", "fqsl_last_error", "fqsl_field_create", "fqsl_field_destroy",
           "fqsl_qmap_plane", "fqsl_qmap_volume", "fqsl_twist", "fqsl_field_check", "fqsl_field_set_timing",
           "fqsl_field_times", "fqsl_field_update", "fqsl_qmap_plane_static", "fqsl_batch_create", "fqsl_batch_run",
           "fqsl_batch_destroy", "fqsl_backward", "fqsl_loss_logq_tw", "fqsl_tape_export",
           "fqsl_tape_destroy", "fqsl_field_create_rect", "fqsl_debug_alloc_cap")
STATIC_MAX_SEEDS = 65536


class FqslError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("fqsl status %d: %s" % (status, msg))
        self.status = status


class Params(C.Structure):
    _fields_ = [("method", C.c_int), ("gradb_way", C.c_int), ("precision", C.c_int), ("refill_lanes", C.c_int),
                ("tol", C.c_double), ("h0", C.c_double), ("h_min", C.c_double), ("h_max", C.c_double),
                ("max_steps", C.c_longlong), ("rot_thresh", C.c_double), ("tol_exp", C.c_double),
                ("graze", C.c_double), ("eps_way2", C.c_double), ("sync_dirs", C.c_int), ("chunk_tiles", C.c_int),
                ("blocks_per_sm", C.c_int), ("tape", C.c_int), ("tape_chunk", C.c_int),
                ("reverse_precision", C.c_int), ("qperp", C.c_int), ("scheme", C.c_int), ("step", C.c_double),
                ("step_min", C.c_double)]


class Plane(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("u", C.c_double * 3), ("v", C.c_double * 3), ("nu", C.c_longlong),
                ("nv", C.c_longlong)]


class Out(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("Q", "Tw", "length", "r1", "r2", "face1", "face2", "status", "steps")]


def load(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("libfqsl.so not found at %s: build it with __graft_entry__.build() "
                          "(the fqsl library has no CPU fallback)" % path)
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.fqsl_params_default.argtypes = [C.POINTER(Params)]
    lib.fqsl_params_default.restype = None
    lib.fqsl_version.restype = C.c_char_p
    lib.fqsl_last_error.restype = C.c_char_p
    lib.fqsl_field_create.argtypes = [P, C.c_int, C.c_longlong, C.c_longlong, C.c_longlong, P, P, C.c_uint, P,
                                      C.POINTER(P)]
    lib.fqsl_field_create_rect.argtypes = [P, C.c_int, C.c_longlong, C.c_longlong, C.c_longlong, P, P, P, C.c_uint,
                                           P, C.POINTER(P)]
    lib.fqsl_field_destroy.argtypes = [P]
    lib.fqsl_qmap_plane.argtypes = [P, P, P, P, C.c_longlong, C.c_longlong, C.POINTER(Params), C.POINTER(Out),
                                    C.POINTER(P), P]
    lib.fqsl_qmap_plane_static.argtypes = [P, P, P, P, C.c_longlong, C.c_longlong, C.POINTER(Params),
                                           C.POINTER(Out), P]
    lib.fqsl_qmap_volume.argtypes = [P, P, P, C.c_longlong, C.c_longlong, C.c_longlong, C.POINTER(Params),
                                     C.POINTER(Out), C.POINTER(P), P]
    lib.fqsl_twist.argtypes = [P, P, C.c_longlong, C.POINTER(Params), C.POINTER(Out), P]
    lib.fqsl_field_check.argtypes = [P, P]
    lib.fqsl_field_set_timing.argtypes = [P, C.c_int]
    lib.fqsl_batch_create.argtypes = [P, P, P, C.c_int, C.POINTER(Params), C.POINTER(P)]
    lib.fqsl_batch_run.argtypes = [P, P]
    lib.fqsl_batch_destroy.argtypes = [P]
    lib.fqsl_field_update.argtypes = [P, P, C.c_int, P]
    lib.fqsl_field_times.argtypes = [P, C.POINTER(C.c_float * 3)]
    lib.fqsl_backward.argtypes = [P, P, P, P, P, C.c_int, P]
    lib.fqsl_tape_export.argtypes = [P, C.c_int, P, P, P, P, P]
    lib.fqsl_tape_destroy.argtypes = [P]
    lib.fqsl_loss_logq_tw.argtypes = [C.c_longlong, P, P, P, P, P, C.c_double, P, P, P, P, P]
    lib.fqsl_debug_alloc_cap.argtypes = [C.c_ulonglong]
    for name in EXPORTS:
        if name not in ("fqsl_params_default", "fqsl_version", "fqsl_last_error", "fqsl_debug_alloc_cap"):
            getattr(lib, name).restype = C.c_int
    lib.fqsl_debug_alloc_cap.restype = None
    return lib


_lib = load()


def version() -> str:
    return _lib.fqsl_version().decode()


def debug_alloc_cap(nbytes: int) -> None:
    """Testing aid (fqsl_debug_alloc_cap): later device allocations of the
    library larger than ``nbytes`` fail as out of memory (FqslError status 3);
    0 removes the cap."""
    _lib.fqsl_debug_alloc_cap(int(nbytes))


def _check(status):
    if status != 0:
        raise FqslError(status, _lib.fqsl_last_error().decode())


def params(**kw) -> Params:
    """fqsl_params with the library defaults, overridden by keyword
    (method, gradb_way, precision ('f32'/'f64'/'f32acc64' or 0/1/2), tol, h0, h_min, h_max,
    max_steps, rot_thresh, tol_exp, graze, eps_way2, qperp (Method II Q_perp), scheme (0 RKF45, 1
    fixed-step 3/8-rule RK4) with step and step_min, scheduling knobs, and for the adjoint tape,
    tape_chunk, reverse_precision)."""
    p = Params()
    _lib.fqsl_params_default(C.byref(p))
    for k, v in kw.items():
        if k in ("precision", "reverse_precision") and isinstance(v, str):
            v = {"f32": F32, "f64": F64, "f32acc64": F32_ACC64}[v]
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _vec3(v):
    return (C.c_double * 3)(*[float(x) for x in v])


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Field:
    """A field handle: B (torch CUDA tensor (nz, ny, nx, 3), float32 or float64)
    packed with its curl into node records (pack: 'f32', 'f64' or both, plus
    'gradb' for the grad(B/|B|) grid of Method II way 1). The grid is uniform
    (origin, spacing) or stretched (coords = the x, y, z node coordinates,
    fqsl_field_create_rect)."""

    def __init__(self, B: torch.Tensor, origin=None, spacing=None, pack=("f32", "f64"), stream=None, coords=None):
        if not (isinstance(B, torch.Tensor) and B.is_cuda and B.dim() == 4 and B.shape[-1] == 3):
            raise ValueError("B must be a CUDA tensor of shape (nz, ny, nx, 3)")
        if B.dtype not in (torch.float32, torch.float64):
            raise ValueError("B must be float32 or float64")
        if (coords is None) == (origin is None or spacing is None):
            raise ValueError("give either origin and spacing (uniform grid) or coords (stretched grid)")
        B = B.contiguous()
        nz, ny, nx, _ = B.shape
        flags = ((PACK_F32 if "f32" in pack else 0) | (PACK_F64 if "f64" in pack else 0) |
                 (PACK_GRADB if "gradb" in pack else 0))
        h = C.c_void_p()
        bt = F32 if B.dtype == torch.float32 else F64
        if coords is None:
            _check(_lib.fqsl_field_create(C.c_void_p(B.data_ptr()), bt, nx, ny, nz, _vec3(origin), _vec3(spacing),
                                          flags, _stream(stream), C.byref(h)))
            self.origin = tuple(float(v) for v in origin)
            self.spacing = tuple(float(v) for v in spacing)
            self.coords = None
        else:
            xs = [(C.c_double * len(c))(*[float(v) for v in c]) for c in coords]
            if tuple(len(c) for c in coords) != (nx, ny, nz):
                raise ValueError("coords must hold nx, ny, nz node coordinates")
            _check(_lib.fqsl_field_create_rect(C.c_void_p(B.data_ptr()), bt, nx, ny, nz, xs[0], xs[1], xs[2], flags,
                                               _stream(stream), C.byref(h)))
            self.coords = tuple(tuple(float(v) for v in c) for c in coords)
            self.origin = tuple(c[0] for c in self.coords)
            self.spacing = None
        self._h = h
        self.n = (nx, ny, nz)
        self._keep = B  # the packing kernel reads B asynchronously
        self._free_tapes = []  # handles of released pooled tapes (see Tape)

    @property
    def handle(self):
        return self._h

    def check(self, stream=None):
        _check(_lib.fqsl_field_check(self._h, _stream(stream)))

    def update(self, B: torch.Tensor, stream=None):
        """Repack a new B of the same shape (a later snapshot) into this handle."""
        if not (isinstance(B, torch.Tensor) and B.is_cuda and tuple(B.shape) == (self.n[2], self.n[1], self.n[0], 3)):
            raise ValueError("B must be a CUDA tensor of shape (nz, ny, nx, 3) matching the field")
        B = B.contiguous()
        _check(_lib.fqsl_field_update(self._h, C.c_void_p(B.data_ptr()), F32 if B.dtype == torch.float32 else F64,
                                      _stream(stream)))
        self._keep = B
        self._packed_from = None  # QTwPlane sets it after its own update

    def set_timing(self, enable: bool = True):
        """Record CUDA events around this field's kernels on each call's stream."""
        _check(_lib.fqsl_field_set_timing(self._h, 1 if enable else 0))

    def times(self):
        """(tracer ms, rotated-extra tracer ms, assembly ms) of the last call."""
        ms = (C.c_float * 3)()
        _check(_lib.fqsl_field_times(self._h, C.byref(ms)))
        return tuple(float(v) for v in ms)

    def close(self):
        t = getattr(self, "_default_tape", None)
        if t is not None:
            t.close()
            self._default_tape = None
        for h in getattr(self, "_free_tapes", ()):
            _lib.fqsl_tape_destroy(h)
        self._free_tapes = []
        if getattr(self, "_h", None):
            _lib.fqsl_field_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def alloc_out(n: int, device="cuda", q=True):
    """Device output buffers for n seeds."""
    f64 = dict(dtype=torch.float64, device=device)
    return dict(Q=torch.empty(n, **f64) if q else None, Tw=torch.empty(n, **f64), length=torch.empty(n, **f64),
                r1=torch.empty((n, 3), **f64), r2=torch.empty((n, 3), **f64),
                face1=torch.empty(n, dtype=torch.int8, device=device),
                face2=torch.empty(n, dtype=torch.int8, device=device),
                status=torch.empty(n, dtype=torch.uint8, device=device),
                steps=torch.empty(n, dtype=torch.int32, device=device))


def _out_struct(out):
    o = Out()
    for name, _ in Out._fields_:
        t = out.get(name)
        setattr(o, name, None if t is None else t.data_ptr())
    return o


class Tape:
    """A taped map (fqsl_tape): made by the first qmap_plane / qmap_volume call
    with params(tape=1) that is given it, re-recorded by later ones, read by
    backward() and tape_export(); its device memory is released by close().
    A tape made with ``pool=field`` hands its C handle (and the device memory
    it holds) back to that field when it is garbage-collected, for the next
    pooled tape to reuse; the field releases pooled handles when it closes."""

    def __init__(self, pool=None):
        self._h = C.c_void_p()
        self._pool = pool
        if pool is not None and getattr(pool, "_free_tapes", None):
            self._h = pool._free_tapes.pop()

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("the tape holds no map yet")
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib.fqsl_tape_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            pool = getattr(self, "_pool", None)
            if self._h and pool is not None and getattr(pool, "_h", None):
                pool._free_tapes.append(self._h)  # reused by the field's next pooled tape
                self._h = C.c_void_p()
            else:
                self.close()
        except Exception:
            pass


def _tape_arg(field, p, tape):
    """The tape of a taped call: the one given, else the field's own default
    tape (made once, re-recorded by every taped call given no tape, so that a
    loop reuses its device memory). The field remembers the last tape used for
    backward() and tape_export() called without one."""
    if not p.tape:
        return None, None
    t = tape
    if t is None:
        t = getattr(field, "_default_tape", None)
        if t is None:
            t = field._default_tape = Tape()
    field.last_tape = t
    return t, C.byref(t._h)


def qmap_plane(field: Field, origin, u, v, nu: int, nv: int, p: Params | None = None, out=None, stream=None,
               tape: Tape | None = None):
    """Q, Tw, length, footpoints, faces, status, steps on the plane lattice
    origin + (i+1/2) u + (j+1/2) v (index i + nu j). With params(tape=1) the
    map is also recorded into ``tape`` (if None, the field's default tape),
    which becomes ``field.last_tape``."""
    p = p or params()
    out = out or alloc_out(nu * nv)
    _, tp = _tape_arg(field, p, tape)
    _check(_lib.fqsl_qmap_plane(field.handle, _vec3(origin), _vec3(u), _vec3(v), nu, nv, C.byref(p),
                                C.byref(_out_struct(out)), tp, _stream(stream)))
    return out


def qmap_plane_static(field: Field, origin, u, v, nu: int, nv: int, p: Params | None = None, out=None,
                      stream=None):
    """qmap_plane through fqsl_qmap_plane_static: the library allocates no device
    memory for the call (its scratch is a fixed static array; nu*nv <=
    STATIC_MAX_SEEDS; calls must not overlap on the GPU). The output buffers
    are the caller's: pass ``out`` to avoid allocating them here."""
    p = p or params()
    out = out or alloc_out(nu * nv)
    _check(_lib.fqsl_qmap_plane_static(field.handle, _vec3(origin), _vec3(u), _vec3(v), nu, nv, C.byref(p),
                                       C.byref(_out_struct(out)), _stream(stream)))
    return out


def qmap_volume(field: Field, origin, step, nx: int, ny: int, nz: int, p: Params | None = None, out=None,
                stream=None, tape: Tape | None = None):
    """The same on the volume lattice origin + (i+1/2, j+1/2, k+1/2) * step."""
    p = p or params()
    out = out or alloc_out(nx * ny * nz)
    _, tp = _tape_arg(field, p, tape)
    _check(_lib.fqsl_qmap_volume(field.handle, _vec3(origin), _vec3(step), nx, ny, nz, C.byref(p),
                                 C.byref(_out_struct(out)), tp, _stream(stream)))
    return out


def twist(field: Field, seeds: torch.Tensor, p: Params | None = None, out=None, stream=None):
    """Tw, length, footpoints for explicit seeds (CUDA float64 tensor (n, 3))."""
    p = p or params()
    seeds = seeds.to(torch.float64).contiguous()
    n = seeds.shape[0]
    out = out or alloc_out(n, q=False)
    _check(_lib.fqsl_twist(field.handle, C.c_void_p(seeds.data_ptr()), n, C.byref(p), C.byref(_out_struct(out)),
                           _stream(stream)))
    return out


class Batch:
    """A batch plan: entries (field, plane) of uneven sizes mapped by one set of
    launches (fqsl_batch_*). ``planes`` are dicts with origin, u, v, nu, nv.
    Output buffers are allocated here (``outs[k]``) unless given. ``run()`` only
    launches kernels on the stream, so it can be captured in a CUDA graph
    (``graph()``)."""

    def __init__(self, fields, planes, p: Params | None = None, outs=None, device="cuda"):
        self.p = p or params()
        self.fields = list(fields)
        self.planes = [dict(pl) for pl in planes]
        n = len(self.fields)
        self.outs = outs or [alloc_out(pl["nu"] * pl["nv"], device=device) for pl in self.planes]
        F = (C.c_void_p * n)(*[f.handle.value for f in self.fields])
        PL = (Plane * n)()
        for k, pl in enumerate(self.planes):
            PL[k].origin = (C.c_double * 3)(*map(float, pl["origin"]))
            PL[k].u = (C.c_double * 3)(*map(float, pl["u"]))
            PL[k].v = (C.c_double * 3)(*map(float, pl["v"]))
            PL[k].nu = int(pl["nu"])
            PL[k].nv = int(pl["nv"])
        O = (Out * n)(*[_out_struct(o) for o in self.outs])
        h = C.c_void_p()
        _check(_lib.fqsl_batch_create(F, PL, O, n, C.byref(self.p), C.byref(h)))
        self._h = h

    def run(self, stream=None):
        _check(_lib.fqsl_batch_run(self._h, _stream(stream)))
        return self.outs

    def graph(self, warmup: int = 1):
        """Capture run() into a torch CUDA graph; replay it with .replay()."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.run()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        return g

    def close(self):
        if getattr(self, "_h", None):
            _lib.fqsl_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _tape_of(field, tape):
    t = tape if tape is not None else getattr(field, "last_tape", None)
    if t is None:
        raise RuntimeError("no taped map: trace one with params(tape=1) first")
    return t


def backward(field: Field, dQ=None, dTw=None, dB=None, dtype=None, stream=None, tape: Tape | None = None):
    """Accumulate (d(Q,Tw)/dB)^T (dQ, dTw) of the taped map in ``tape``
    (default: the field's last taped map) into dB (a B-shaped CUDA tensor;
    allocated as zeros of ``dtype``, default float32, when not given). dQ, dTw:
    CUDA float64 tensors of the map's seed count, or None."""
    t = _tape_of(field, tape)
    nx, ny, nz = field.n
    if dB is None:
        dB = torch.zeros((nz, ny, nx, 3), dtype=dtype or torch.float32, device="cuda")
    if not (dB.is_cuda and dB.is_contiguous() and tuple(dB.shape) == (nz, ny, nx, 3)):
        raise ValueError("dB must be a contiguous CUDA tensor of shape (nz, ny, nx, 3)")
    if dB.dtype not in (torch.float32, torch.float64):
        raise ValueError("dB must be float32 or float64")
    dQ = None if dQ is None else dQ.to(torch.float64).contiguous()
    dTw = None if dTw is None else dTw.to(torch.float64).contiguous()
    _check(_lib.fqsl_backward(field.handle, t.handle, _ptr(dQ), _ptr(dTw), C.c_void_p(dB.data_ptr()),
                              F32 if dB.dtype == torch.float32 else F64, _stream(stream)))
    return dB


def tape_export(field: Field, n_seeds: int, cap: int = 4096, stream=None, tape: Tape | None = None):
    """The step sequence of a taped map (default: the field's last;
    fqsl_tape_export): dict of CUDA tensors nsteps (2n), code (2n), hx (2n),
    h (2n, cap); half-line 2 s + e is end e + 1 of seed s."""
    t = _tape_of(field, tape)
    dev = "cuda"
    m = 2 * n_seeds
    out = dict(nsteps=torch.empty(m, dtype=torch.int32, device=dev), code=torch.empty(m, dtype=torch.int32, device=dev),
               hx=torch.empty(m, dtype=torch.float64, device=dev),
               h=torch.zeros((m, max(cap, 1)), dtype=torch.float64, device=dev))
    _check(_lib.fqsl_tape_export(t.handle, cap, _ptr(out["nsteps"]), _ptr(out["code"]), _ptr(out["hx"]),
                                 _ptr(out["h"]), _stream(stream)))
    return out


def loss_logq_tw(Q, Tw, Q_target, Tw_target, status=None, w_tw: float = 0.1, stream=None, out=None):
    """mean over usable seeds of (log10 Q - log10 Q_t)^2 + w_tw (Tw - Tw_t)^2 and
    its gradient (fqsl_loss_logq_tw). Returns (loss (0-d CUDA tensor), dQ, dTw)."""
    n = Q.numel()
    dev = Q.device
    if out is None:
        out = dict(sums=torch.empty(2, dtype=torch.float64, device=dev),
                   loss=torch.empty((), dtype=torch.float64, device=dev),
                   dQ=torch.empty(n, dtype=torch.float64, device=dev),
                   dTw=torch.empty(n, dtype=torch.float64, device=dev))
    args = [t.contiguous() for t in (Q, Tw, Q_target, Tw_target)]
    if any(t.dtype != torch.float64 for t in args):
        raise ValueError("Q, Tw and the targets must be float64")
    st = None if status is None else status.contiguous()
    _check(_lib.fqsl_loss_logq_tw(n, *[_ptr(t) for t in args], _ptr(st), float(w_tw), _ptr(out["sums"]),
                                  _ptr(out["loss"]), _ptr(out["dQ"]), _ptr(out["dTw"]), _stream(stream)))
    return out["loss"], out["dQ"], out["dTw"]


class QTwPlane(torch.autograd.Function):
    """(Q, Tw) of a plane map as a differentiable function of B:
    ``Q, Tw = QTwPlane.apply(B, field, origin, u, v, nu, nv, p)``. The forward
    packs B into ``field`` (unless the field already holds this very tensor
    unchanged) and traces the map into a tape of its own; the backward runs
    fqsl_backward on that tape (frozen step sequence; Method I). Several maps of
    one field (other planes) can therefore sit in one graph. Q of rotated or NaN
    seeds carries no gradient."""

    @staticmethod
    def forward(ctx, B, field, origin, u, v, nu, nv, p=None):
        p = p or params()
        q = Params.from_buffer_copy(p)
        q.tape = 1
        key = (B.data_ptr(), B._version, tuple(B.shape), B.dtype)
        if getattr(field, "_packed_from", None) != key:
            field.update(B.detach())
            field._packed_from = key
        ctx.tape = Tape(pool=field)  # a released graph's tape is reused by the next forward
        prev = getattr(field, "last_tape", None)
        out = qmap_plane(field, origin, u, v, nu, nv, q, tape=ctx.tape)
        field.last_tape = prev  # only the graph holds this tape
        ctx.field = field
        ctx.b_dtype = B.dtype
        return out["Q"], out["Tw"]

    @staticmethod
    def backward(ctx, gQ, gTw):
        dB = backward(ctx.field, gQ, gTw, dtype=ctx.b_dtype, tape=ctx.tape)
        return dB, None, None, None, None, None, None, None
