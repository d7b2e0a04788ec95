"""FP64 CPU adjoint oracle -- TEST INFRASTRUCTURE ONLY.

Reverse (and tangent-linear) derivatives of the plane-lattice Q and Tw maps
(Method I) with respect to the field cube B, in plain PyTorch CPU float64.

The C oracle traces every lattice line once and records its accepted steps
(``oracle_lattice_log``): the step size of each accepted RKF45 step, and how
each direction ended (exit step onto a face, the same with the point clamped
into the box, or the chord fallback after an exiting step of a given size).
This module replays exactly that step sequence with the step sizes, exit faces
and exit kinds frozen, recomputing from the leaf tensor B everything else: the
curl grid, every stage position and RHS value (Sec. 2.2 Eq. interp and the
index-space line equation of Sec. 2.1 / 2.3), the exit-step length (distance
to the face), the chord parameter, the footpoints, Tw (Eq. tw), Bn at the
seed and at both ends (Eq. Bn1) and Method I's Q (Eqs. D+-2, D+-3, Q+-), with
the finite-difference stencils the oracle chose (reading R8). Autograd (reverse
mode) and forward-mode AD then give d(output)/dB of this frozen-sequence map,
the discrete adjoint the CUDA reverse sweep implements.

Only the tests and the benchmark's CPU leg use this module.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import BAD, ROTATED, _coords, _f64, _grid_args, _p, curl, is_rect, lib, params, plane

# Fehlberg 4(5) stage matrix and 4th-order weights (the propagated solution)
_A = [[], [1 / 4], [3 / 32, 9 / 32], [1932 / 2197, -7200 / 2197, 7296 / 2197],
      [439 / 216, -8.0, 3680 / 513, -845 / 4104], [-8 / 27, 2.0, -3544 / 2565, 1859 / 4104, -11 / 40]]
_B4 = [25 / 216, 0.0, 1408 / 2565, 2197 / 4104, -1 / 5, 0.0]
# Kutta's 3/8 rule (the fixed-step scheme, reading R18)
_A38 = [[], [1 / 3], [-1 / 3, 1.0], [1.0, -1.0, 1.0]]
_B38 = [1 / 8, 3 / 8, 3 / 8, 1 / 8]

# step-record codes of oracle_lattice_log
START, STEP, EXIT, EXIT_CLAMPED, CHORD = 99, 0, 16, 40, 48


def lattice_log(B, grid, origin, u, v, nu, nv, p=None, cap=8192, J=None, which=None, extra=True):
    """Trace every line of the plane lattice (or only the lattice indices in
    ``which``, in that order) once with the C oracle; return their step
    records and outcomes (numpy arrays, one row per traced line). With extra,
    the four extra lines of each rotated-S0 seed are recorded too (x* arrays,
    4 per row)."""
    p = p or params()
    B = _f64(B)
    J = _f64(curl(B, grid) if J is None else J)
    wh = None if which is None else np.ascontiguousarray(which, dtype=np.int64)
    m = nu * nv if wh is None else len(wh)
    out = dict(h=np.zeros((m, cap)), code=np.zeros((m, cap), np.int32), n=np.zeros(m, np.int32),
               s0=np.zeros(m), tol=np.zeros(m), bn0=np.zeros(m), ends=np.zeros((m, 2, 11)),
               faces=np.zeros((m, 2), np.int32), status=np.zeros(m, np.int32))
    if extra:
        out.update(xh=np.zeros((m, 4, cap)), xcode=np.zeros((m, 4, cap), np.int32), xn=np.zeros((m, 4), np.int32),
                   xs0=np.zeros((m, 4)), xfaces=np.zeros((m, 4, 2), np.int32), xstatus=np.zeros((m, 4), np.int32))
    X = (lambda k: _p(out[k]) if extra else None)  # noqa: E731
    lo = np.array(origin, float)
    a1, a2 = np.array(u, float), np.array(v, float)
    ln = np.array([nu, nv], np.int64)
    L = lib()
    tail = (_p(lo), _p(a1), _p(a2), _p(ln), C.byref(p), C.c_int(cap), _p(out["h"]), _p(out["code"]), _p(out["n"]),
            _p(out["s0"]), _p(out["tol"]), _p(out["bn0"]), _p(out["ends"]), _p(out["faces"]), _p(out["status"]),
            _p(wh), C.c_longlong(0 if wh is None else len(wh)),
            X("xh"), X("xcode"), X("xn"), X("xs0"), X("xfaces"), X("xstatus"))
    if is_rect(grid):
        # stretched grid (reading R16): the recorded ends are physical positions
        n = np.array(grid.n, dtype=np.int64)
        rc = L.oracle_lattice_log_rect(_p(B), _p(J), _p(n), _p(_coords(grid)), *tail)
    else:
        n, o, d = _grid_args(grid)
        L.oracle_lattice_log.restype = C.c_int
        rc = L.oracle_lattice_log(_p(B), _p(J), _p(n), _p(o), _p(d), *tail)
    if rc:
        raise ValueError("oracle_lattice_log: error %d" % rc)
    if np.any(out["n"] < 0) or (extra and np.any(out["xn"] < 0)):
        raise ValueError("step record overflow: raise cap")
    out["scheme"] = int(p.scheme)
    return out


def curl_t(B, spacing):
    """curl B at the nodes (B of shape (nz, ny, nx, 3)): 2nd-order central
    differences inside, 2nd-order one-sided on the faces, first order on an
    axis of 2 nodes -- the stencils of the oracle's curl grid, in torch."""
    def deriv(f, dim, h):
        n = f.shape[dim]
        s = lambda a, b: f.narrow(dim, a, b - a)  # noqa: E731
        if n == 2:
            g = (s(1, 2) - s(0, 1)) / h
            return torch.cat([g, g], dim=dim)
        first = (-3.0 * s(0, 1) + 4.0 * s(1, 2) - s(2, 3)) / (2.0 * h)
        mid = (s(2, n) - s(0, n - 2)) / (2.0 * h)
        last = (3.0 * s(n - 1, n) - 4.0 * s(n - 2, n - 1) + s(n - 3, n - 2)) / (2.0 * h)
        return torch.cat([first, mid, last], dim=dim)

    dx, dy, dz = spacing
    Bx, By, Bz = B[..., 0], B[..., 1], B[..., 2]
    # tensor dims: 0 = z, 1 = y, 2 = x
    Jx = deriv(Bz, 1, dy) - deriv(By, 0, dz)
    Jy = deriv(Bx, 0, dz) - deriv(Bz, 2, dx)
    Jz = deriv(By, 2, dx) - deriv(Bx, 1, dy)
    return torch.stack([Jx, Jy, Jz], dim=-1)


def _deriv_rect(f, dim, X):
    """d f/d x along tensor dim with node coordinates X (reading R16): the
    derivative of the quadratic through three neighbouring nodes, one-sided at
    the ends, first order on an axis of 2 nodes."""
    X = np.asarray(X, dtype=np.float64)
    n = f.shape[dim]
    s = lambda a, b: f.narrow(dim, a, b - a)  # noqa: E731

    def col(v):
        shape = [1] * f.dim()
        shape[dim] = -1
        return torch.as_tensor(np.atleast_1d(v), dtype=torch.float64).reshape(shape)
    if n == 2:
        g = (s(1, 2) - s(0, 1)) / float(X[1] - X[0])
        return torch.cat([g, g], dim=dim)
    h1, h2 = X[1] - X[0], X[2] - X[1]
    first = (-(2.0 * h1 + h2) / (h1 * (h1 + h2)) * s(0, 1) + (h1 + h2) / (h1 * h2) * s(1, 2)
             - h1 / (h2 * (h1 + h2)) * s(2, 3))
    a, b = X[1:-1] - X[:-2], X[2:] - X[1:-1]
    mid = (col(-b / (a * (a + b))) * s(0, n - 2) + col((b - a) / (a * b)) * s(1, n - 1)
           + col(a / (b * (a + b))) * s(2, n))
    h1, h2 = X[n - 2] - X[n - 3], X[n - 1] - X[n - 2]
    last = (h2 / (h1 * (h1 + h2)) * s(n - 3, n - 2) - (h1 + h2) / (h1 * h2) * s(n - 2, n - 1)
            + (h1 + 2.0 * h2) / (h2 * (h1 + h2)) * s(n - 1, n))
    return torch.cat([first, mid, last], dim=dim)


def curl_t_rect(B, coords):
    """curl B at the nodes of a stretched grid (B of shape (nz, ny, nx, 3)), with
    the three-point stencils of a non-uniform axis, in torch."""
    xs, ys, zs = coords
    Bx, By, Bz = B[..., 0], B[..., 1], B[..., 2]
    Jx = _deriv_rect(Bz, 1, ys) - _deriv_rect(By, 0, zs)
    Jy = _deriv_rect(Bx, 0, zs) - _deriv_rect(Bz, 2, xs)
    Jz = _deriv_rect(By, 2, xs) - _deriv_rect(Bx, 1, ys)
    return torch.stack([Jx, Jy, Jz], dim=-1)


class _Field:
    """B and curl B node values flattened to (nodes, 6), and trilinear
    interpolation at index positions (Sec. 2.2): the cell is the floor of the
    position clamped to [0, n-2] (chosen without a derivative), the weights
    are linear in the position."""

    def __init__(self, Bt, Jt, n, spacing):
        self.n = n
        self.BJ = torch.cat([Bt, Jt], dim=-1).reshape(-1, 6)
        self.d = torch.tensor(spacing, dtype=torch.float64)
        self.cmax = torch.tensor([n[0] - 2, n[1] - 2, n[2] - 2], dtype=torch.float64)
        nx, ny, _ = n
        self.off = [(m, q, p, (p * ny + q) * nx + m) for m in (0, 1) for q in (0, 1) for p in (0, 1)]
        self.lo = torch.zeros(3, dtype=torch.float64)
        self.hi = torch.tensor([n[0] - 1.0, n[1] - 1.0, n[2] - 1.0], dtype=torch.float64)

    def widths(self, xi):
        return None  # index space: the spacing is part of rhs

    def interp(self, xi):
        nx, ny, _ = self.n
        with torch.no_grad():
            c = torch.nan_to_num(torch.floor(xi), nan=0.0)
            c = torch.minimum(torch.maximum(c, torch.zeros_like(c)), self.cmax)
            ci = c.long()
            base = (ci[:, 2] * ny + ci[:, 1]) * nx + ci[:, 0]
            nodes = torch.stack([base + o for (_, _, _, o) in self.off], dim=1)
        w1 = xi - c
        w0 = 1.0 - w1
        wts = torch.stack([(w1[:, 0] if m else w0[:, 0]) * (w1[:, 1] if q else w0[:, 1]) *
                           (w1[:, 2] if p else w0[:, 2]) for (m, q, p, _) in self.off], dim=1)
        vals = self.BJ[nodes]  # (k, 8, 6)
        out = (wts[:, :, None] * vals).sum(1)
        return out[:, :3], out[:, 3:]

    def rhs(self, xi, sigma, D=None):
        """Index-space line equation: F = sigma bt/|bt| (bt_a = B_a/d_a), and
        the Tw integrand (J.B)/(4 pi B^2) dl/dtau with dl/dtau = |B|/|bt|."""
        Bi, Ji = self.interp(xi)
        bt = Bi / self.d
        nbt = torch.sqrt((bt * bt).sum(-1))
        BB = (Bi * Bi).sum(-1)
        F = sigma[:, None] * bt / nbt[:, None]
        dl = torch.sqrt(BB) / nbt
        dtw = (Ji * Bi).sum(-1) / (4.0 * math.pi * BB) * dl
        return F, dtw


class _RectField:
    """The same on a stretched grid (reading R16): physical positions; the cell
    of a coordinate is the largest i in [0, n-2] with x_i <= x (below x_0, and
    NaN, cell 0), chosen without a derivative; Eq. w0 weights in physical
    coordinates; the line equation dr/dtau = sigma B/|bt| with bt_a = B_a/D_a,
    D the widths of the cell the step starts in."""

    def __init__(self, Bt, Jt, coords):
        self.X = [np.asarray(c, dtype=np.float64) for c in coords]
        self.Xt = [torch.from_numpy(x) for x in self.X]
        self.n = tuple(len(x) for x in self.X)
        self.BJ = torch.cat([Bt, Jt], dim=-1).reshape(-1, 6)
        nx, ny, _ = self.n
        self.off = [(m, q, p, (p * ny + q) * nx + m) for m in (0, 1) for q in (0, 1) for p in (0, 1)]
        self.lo = torch.tensor([x[0] for x in self.X], dtype=torch.float64)
        self.hi = torch.tensor([x[-1] for x in self.X], dtype=torch.float64)

    def cells(self, x):
        with torch.no_grad():
            out = []
            for a in range(3):
                xa = x[:, a].detach().numpy()
                c = np.searchsorted(self.X[a], xa, side="right") - 1
                c = np.where(np.isnan(xa) | ~(xa >= self.X[a][0]), 0, c)
                out.append(np.clip(c, 0, self.n[a] - 2))
            return torch.from_numpy(np.stack(out, axis=1).astype(np.int64))

    def widths(self, x):
        c = self.cells(x)
        return torch.stack([self.Xt[a][c[:, a] + 1] - self.Xt[a][c[:, a]] for a in range(3)], dim=1)

    def interp(self, x):
        nx, ny, _ = self.n
        c = self.cells(x)
        w0 = torch.stack([(self.Xt[a][c[:, a] + 1] - x[:, a]) / (self.Xt[a][c[:, a] + 1] - self.Xt[a][c[:, a]])
                          for a in range(3)], dim=1)
        w1 = 1.0 - w0
        base = (c[:, 2] * ny + c[:, 1]) * nx + c[:, 0]
        nodes = torch.stack([base + o for (_, _, _, o) in self.off], dim=1)
        wts = torch.stack([(w1[:, 0] if m else w0[:, 0]) * (w1[:, 1] if q else w0[:, 1]) *
                           (w1[:, 2] if p else w0[:, 2]) for (m, q, p, _) in self.off], dim=1)
        out = (wts[:, :, None] * self.BJ[nodes]).sum(1)
        return out[:, :3], out[:, 3:]

    def rhs(self, x, sigma, D):
        Bi, Ji = self.interp(x)
        bt = Bi / D
        nbt = torch.sqrt((bt * bt).sum(-1))
        BB = (Bi * Bi).sum(-1)
        F = sigma[:, None] * Bi / nbt[:, None]
        dl = torch.sqrt(BB) / nbt
        dtw = (Ji * Bi).sum(-1) / (4.0 * math.pi * BB) * dl
        return F, dtw


def _rk4(fld, x, h, sig, ax=None, scheme=0):
    """One Fehlberg step of the 4th-order solution from x (scheme 1: one
    3/8-rule step). With ax (face axis per lane) the independent variable is
    that index coordinate (exit step): the RHS is divided by its ax
    component."""
    A, Bw = (_A38, _B38) if scheme == 1 else (_A, _B4)
    D = fld.widths(x)  # stretched grid: the widths of the step's start cell
    ks, ts = [], []
    for s in range(len(Bw)):
        acc = sum(A[s][r] * ks[r] for r in range(s)) if s else torch.zeros_like(x)
        F, dtw = fld.rhs(x + h[:, None] * acc, sig, D)
        if ax is not None:
            fa = F.gather(1, ax[:, None])[:, 0]
            F, dtw = F / fa[:, None], dtw / fa
        ks.append(F)
        ts.append(dtw)
    x4 = x + h[:, None] * sum(Bw[s] * ks[s] for s in range(len(Bw)))
    dtw4 = h * sum(Bw[s] * ts[s] for s in range(len(Bw)))
    return x4, dtw4


def half_lines(log):
    """Split each line's record into its two directions (half-lines 2i, 2i+1,
    i.e. end 1 and end 2): codes and step sizes, padded with code -1."""
    m = len(log["n"])
    seqs = []
    for i in range(m):
        codes, hs = log["code"][i, :log["n"][i]], log["h"][i, :log["n"][i]]
        starts = [k for k in range(len(codes)) if codes[k] == START]
        for e in range(2):
            if e < len(starts):
                k1 = starts[e + 1] if e + 1 < len(starts) else len(codes)
                seqs.append((codes[starts[e] + 1:k1], hs[starts[e] + 1:k1]))
            else:
                seqs.append((np.zeros(0, np.int32), np.zeros(0)))
    T = max((len(c) for c, _ in seqs), default=0)
    code = np.full((2 * m, T), -1, np.int64)
    hh = np.zeros((2 * m, T))
    for k, (c, h) in enumerate(seqs):
        code[k, :len(c)] = c
        hh[k, :len(c)] = h
    return code, hh


def replay(fld, xi0, s0, log):
    """Replay the frozen step sequences from the seeds xi0 (m, 3). Returns the
    end positions (m, 2, 3) in index coordinates and Tw of each direction
    (m, 2). End 1 (half-line 2i) is traced along -s0 B."""
    m = xi0.shape[0]
    scheme = log.get("scheme", 0)
    code, hh = half_lines(log)
    H, T = code.shape
    sig = torch.stack([-s0, s0], dim=1).reshape(H)
    lo, hi = fld.lo, fld.hi
    xi = xi0.repeat_interleave(2, dim=0)
    tw = torch.zeros(H, dtype=torch.float64)
    for t in range(T):
        ct = code[:, t]
        # accepted steps inside the box
        i_n = np.nonzero(ct == STEP)[0]
        if len(i_n):
            idx = torch.from_numpy(i_n)
            x4, d4 = _rk4(fld, xi[idx], torch.from_numpy(hh[i_n, t]), sig[idx], scheme=scheme)
            xi = xi.index_put((idx,), x4)
            tw = tw.index_put((idx,), tw[idx] + d4)
        # exit steps (independent variable = face-normal coordinate, Sec. 2.1)
        i_e = np.nonzero(((ct >= EXIT) & (ct < EXIT + 6)) | ((ct >= EXIT_CLAMPED) & (ct < EXIT_CLAMPED + 6)))[0]
        if len(i_e):
            idx = torch.from_numpy(i_e)
            face = torch.from_numpy(np.where(ct[i_e] >= EXIT_CLAMPED, ct[i_e] - EXIT_CLAMPED, ct[i_e] - EXIT))
            ax = face // 2
            target = torch.where(face % 2 == 1, hi[ax], lo[ax])
            x = xi[idx]
            delta = target - x.gather(1, ax[:, None])[:, 0]
            xe, de = _rk4(fld, x, delta, sig[idx], ax, scheme=scheme)
            onehot = torch.nn.functional.one_hot(ax, 3).to(torch.bool)
            xe = torch.where(onehot, target[:, None], xe)
            xe = torch.minimum(torch.maximum(xe, lo), hi)  # the clamp of code 40+
            xi = xi.index_put((idx,), xe)
            tw = tw.index_put((idx,), tw[idx] + de)
        # chord fallback after an exiting step of size h
        i_c = np.nonzero((ct >= CHORD) & (ct < CHORD + 6))[0]
        if len(i_c):
            idx = torch.from_numpy(i_c)
            face = torch.from_numpy(ct[i_c] - CHORD)
            ax = face // 2
            target = torch.where(face % 2 == 1, hi[ax], lo[ax])
            x = xi[idx]
            x4, d4 = _rk4(fld, x, torch.from_numpy(hh[i_c, t]), sig[idx], scheme=scheme)
            xa, x4a = x.gather(1, ax[:, None])[:, 0], x4.gather(1, ax[:, None])[:, 0]
            t0 = (target - xa) / (x4a - xa)
            onehot = torch.nn.functional.one_hot(ax, 3).to(torch.bool)
            xc = torch.where(onehot, target[:, None], x + t0[:, None] * (x4 - x))
            xi = xi.index_put((idx,), xc)
            tw = tw.index_put((idx,), tw[idx] + t0 * d4)
    return xi.reshape(m, 2, 3), tw.reshape(m, 2)


def stencils(faces, status, centres, neighbours, steps):
    """Method I difference coefficients (reading R8) chosen from the traced
    faces: for target t with centre row centres[t], neighbour rows
    neighbours[t] = (+u, -u, +v, -v) (None off the lattice) and lattice steps
    steps[t] = (du, dv), a list of (target, end, lattice axis, row,
    coefficient) with J_e[r][c](target) = sum coefficient * face coordinate r
    of that row's end e; and the targets left MIXED."""
    ok = (status & BAD) == 0
    entries = []
    mixed = np.zeros(len(centres), bool)
    for t, rs in enumerate(centres):
        if not ok[rs]:
            continue
        for e in range(2):
            fe = faces[rs, e]
            for c in range(2):
                dl = steps[t][c]

                def usable(k):
                    return k if k is not None and ok[k] and faces[k, e] == fe else None
                kp, km = usable(neighbours[t][2 * c]), usable(neighbours[t][2 * c + 1])
                if kp is not None and km is not None:
                    entries += [(t, e, c, kp, 0.5 / dl), (t, e, c, km, -0.5 / dl)]
                elif kp is not None:
                    entries += [(t, e, c, kp, 1.0 / dl), (t, e, c, rs, -1.0 / dl)]
                elif km is not None:
                    entries += [(t, e, c, rs, 1.0 / dl), (t, e, c, km, -1.0 / dl)]
                else:
                    mixed[t] = True
    return entries, mixed


_FACE_AXES = {0: (1, 2), 1: (0, 2), 2: (0, 1)}


def seeds_index(grid, origin, u, v, nu, nv):
    """Lattice seeds o + (i+1/2) u + (j+1/2) v, i fastest, in state
    coordinates: index space on a uniform grid, physical on a stretched one."""
    ii = np.arange(nu * nv) % nu
    jj = np.arange(nu * nv) // nu
    r0 = (np.asarray(origin, float)[None] + (ii + 0.5)[:, None] * np.asarray(u, float)[None]) + \
        (jj + 0.5)[:, None] * np.asarray(v, float)[None]
    if is_rect(grid):
        return r0
    return (r0 - np.asarray(grid.origin, float)) / np.asarray(grid.spacing, float)


def neighbourhood(seeds, nu, nv):
    """The seeds and their lattice neighbours (the lines Method I differences
    use), sorted."""
    out = set()
    for s in np.asarray(seeds).ravel():
        i, j = int(s) % nu, int(s) // nu
        for di, dj in ((0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)):
            if 0 <= i + di < nu and 0 <= j + dj < nv:
                out.add(i + di + nu * (j + dj))
    return np.array(sorted(out), dtype=np.int64)


def perp_frame_t(bh, m):
    """Rotated S0 frame (reading R9): u = unit(bhat x e_m), v = bhat x u, with
    the axis m (smallest |bhat_m|) given (chosen without a derivative)."""
    e = torch.nn.functional.one_hot(torch.as_tensor(m), 3).to(bh.dtype)
    t = torch.cross(bh, e, dim=-1)
    uu = t / torch.sqrt((t * t).sum(-1, keepdim=True))
    return uu, torch.cross(bh, uu, dim=-1)


def qmap_t(Bt, grid, origin, u, v, nu, nv, log, lines=None, targets=None):
    """Q and Tw (differentiable in the tensor Bt) from the frozen step
    sequence in log. ``lines``: the lattice indices of log's rows (default:
    every seed, in order); ``targets``: the seeds whose Q and Tw are formed
    (default: every seed), each with its lattice neighbours among the lines.
    A rotated-S0 target's Q uses its four extra lines (recorded in log), whose
    seeds follow the frame of B at the seed. Returns (Q, Tw, usable mask, end
    positions of the lattice rows)."""
    n = grid.n
    rect = is_rect(grid)
    if rect:
        Jt = curl_t_rect(Bt, grid.coords)
        fld = _RectField(Bt, Jt, grid.coords)
    else:
        Jt = curl_t(Bt, grid.spacing)
        fld = _Field(Bt, Jt, n, grid.spacing)
    m = nu * nv
    lines = np.arange(m) if lines is None else np.asarray(lines, dtype=np.int64)
    targets = lines if targets is None else np.asarray(targets, dtype=np.int64)
    row = {int(l): k for k, l in enumerate(lines)}
    tr = np.array([row[int(t)] for t in targets], dtype=np.int64)
    mr = len(lines)
    faces, status = log["faces"], log["status"]
    good = (status & BAD) == 0
    xi_all = seeds_index(grid, origin, u, v, nu, nv)
    # state -> physical: o + d xi (uniform), the identity (stretched)
    d = np.ones(3) if rect else np.asarray(grid.spacing, float)
    o_np = np.zeros(3) if rect else np.asarray(grid.origin, float)
    n0 = np.cross(np.asarray(u, float), np.asarray(v, float))
    n0 = n0 / np.linalg.norm(n0)
    du, dv = float(np.linalg.norm(u)), float(np.linalg.norm(v))
    drot = min(du, dv)
    xi0 = torch.from_numpy(xi_all[lines])
    s0 = torch.from_numpy(log["s0"])
    B0t, _ = fld.interp(torch.from_numpy(xi_all[targets]))
    nB0 = torch.sqrt((B0t * B0t).sum(-1))
    # rotated targets: their extra lines become rows mr, mr + 1, ...
    rot = [t for t in range(len(targets)) if good[tr[t]] and (status[tr[t]] & ROTATED) and "xn" in log]
    xrows = {}
    xi_x, s0_x, xh, xc, xn, xf, xs = [], [], [], [], [], [], []
    for t in rot:
        rs = tr[t]
        bh = B0t[t] / nB0[t]
        with torch.no_grad():
            mm = int(torch.argmin(torch.abs(bh)))  # lowest index on ties
        uu, vv = perp_frame_t(bh, mm)
        r0 = torch.from_numpy(o_np + d * xi_all[targets[t]])
        for q in range(4):
            dirq = uu if q < 2 else vv
            sg = -1.0 if q & 1 else 1.0
            xi_x.append(((r0 + sg * drot * dirq) - torch.from_numpy(o_np)) / torch.from_numpy(d))
            s0_x.append(log["xs0"][rs, q])
            xh.append(log["xh"][rs, q])
            xc.append(log["xcode"][rs, q])
            xn.append(log["xn"][rs, q])
            xf.append(log["xfaces"][rs, q])
            xs.append(log["xstatus"][rs, q])
            xrows[(t, q)] = mr + len(xi_x) - 1
    if xi_x:
        rlog = dict(h=np.concatenate([log["h"], np.stack(xh)]), code=np.concatenate([log["code"], np.stack(xc)]),
                    n=np.concatenate([log["n"], np.array(xn, np.int32)]), scheme=log.get("scheme", 0))
        xi0 = torch.cat([xi0, torch.stack(xi_x)])
        s0 = torch.cat([s0, torch.tensor(s0_x, dtype=torch.float64)])
        faces = np.concatenate([faces, np.stack(xf)])
        status = np.concatenate([status, np.array(xs, np.int32)])
    else:
        rlog = log
    xi, tw = replay(fld, xi0, s0, rlog)
    nrows = xi.shape[0]
    phys = torch.from_numpy(o_np) + torch.from_numpy(d) * xi  # (rows, 2, 3)
    cols = []
    for e in range(2):
        for r in range(2):
            idx = torch.from_numpy(np.array([_FACE_AXES[max(faces[k, e], 0) // 2][r] for k in range(nrows)]))
            cols.append(phys[:, e, :].gather(1, idx[:, None])[:, 0])
    fc = torch.stack(cols, dim=1).reshape(nrows, 2, 2)  # row, end, face coordinate
    neigh, steps = [], []
    for t, sd in enumerate(targets):
        if (t, 0) in xrows:
            neigh.append(tuple(xrows[(t, q)] for q in range(4)))
            steps.append((drot, drot))
        else:
            i, j = int(sd) % nu, int(sd) // nu
            nb = []
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                ii, jj = i + di, j + dj
                nb.append(row.get(ii + nu * jj) if 0 <= ii < nu and 0 <= jj < nv else None)
            neigh.append(tuple(nb))
            steps.append((du, dv))
    entries, mixed = stencils(faces, status, tr, neigh, steps)
    nt = len(targets)
    Jm = torch.zeros((nt, 2, 2, 2), dtype=torch.float64)  # target, end, face row r, lattice axis c
    if entries:
        es = np.array(entries, dtype=float)
        t_i, e_i, c_i, l_i = (torch.from_numpy(es[:, k].astype(np.int64)) for k in range(4))
        coef = torch.from_numpy(es[:, 4])
        for r in range(2):
            Jm = Jm.index_put((t_i, e_i, torch.full_like(t_i, r), c_i), coef * fc[l_i, e_i, r], accumulate=True)
    J1, J2 = Jm[:, 0], Jm[:, 1]
    adj = torch.stack([torch.stack([J1[:, 1, 1], -J1[:, 0, 1]], -1),
                       torch.stack([-J1[:, 1, 0], J1[:, 0, 0]], -1)], 1)
    M = torch.einsum("srk,skc->src", J2, adj)
    norm2 = (M * M).sum((1, 2))
    trt = torch.from_numpy(tr)
    Bend, _ = fld.interp(xi[trt].reshape(-1, 3))
    Bend = Bend.reshape(nt, 2, 3)
    fax = torch.from_numpy(np.maximum(faces[tr], 0) // 2)
    bn1 = Bend[:, 0].gather(1, fax[:, 0:1])[:, 0]
    bn2 = Bend[:, 1].gather(1, fax[:, 1:2])[:, 0]
    rotm = torch.from_numpy((status[tr] & ROTATED) != 0)
    bn0 = torch.where(rotm, nB0, (B0t * torch.from_numpy(n0)).sum(-1))
    Q = norm2 * torch.abs(bn1 * bn2) / (bn0 * bn0)
    usable = torch.from_numpy(good[tr] & ~mixed)
    if "xn" not in log:
        usable = usable & ~rotm
    return Q, tw[trt].sum(1), usable, xi[:mr]


def log_q_tw_loss(Q, Tw, Qt, Twt, usable, wtw=0.1):
    """mean over usable seeds of (log10 Q - log10 Q_t)^2 + wtw (Tw - Tw_t)^2;
    a seed counts when its line is good, not MIXED, and its Q, Q_t are
    positive and finite and Tw, Tw_t finite."""
    qt = torch.as_tensor(np.asarray(Qt, float))
    twt = torch.as_tensor(np.asarray(Twt, float))
    with torch.no_grad():
        use = usable & torch.isfinite(qt) & (qt > 0) & torch.isfinite(Q) & (Q > 0) & torch.isfinite(Tw) & \
            torch.isfinite(twt)
    k = max(int(use.sum()), 1)
    lq = torch.log10(Q[use]) - torch.log10(qt[use])
    return (lq * lq + wtw * (Tw[use] - twt[use]) ** 2).sum() / k, use


def loss_grad(B, grid, origin, u, v, nu, nv, Qt, Twt, p=None, wtw=0.1, log=None):
    """Loss and d(loss)/dB (shape of B) of the frozen-sequence map."""
    p = p or params()
    B = _f64(B)
    log = lattice_log(B, grid, origin, u, v, nu, nv, p) if log is None else log
    Bt = torch.tensor(B, dtype=torch.float64, requires_grad=True)
    Q, Tw, usable, _ = qmap_t(Bt, grid, origin, u, v, nu, nv, log)
    loss, use = log_q_tw_loss(Q, Tw, Qt, Twt, usable, wtw)
    loss.backward()
    return float(loss.detach()), Bt.grad.numpy(), dict(Q=Q.detach().numpy(), Tw=Tw.detach().numpy(), use=use.numpy(),
                                              log=log)


def vjp(B, grid, origin, u, v, nu, nv, wQ, wTw, p=None, log=None):
    """J^T w = d(sum of wQ Q over usable seeds + wTw Tw over good lines)/dB of
    the frozen-sequence map (Q of MIXED seeds is not used; Tw of every line
    without MAXSTEPS, NULL_B or OUTSIDE is)."""
    p = p or params()
    B = _f64(B)
    log = lattice_log(B, grid, origin, u, v, nu, nv, p) if log is None else log
    Bt = torch.tensor(B, dtype=torch.float64, requires_grad=True)
    Q, Tw, usable, _ = qmap_t(Bt, grid, origin, u, v, nu, nv, log)
    good = torch.from_numpy((log["status"] & BAD) == 0)
    wq = torch.as_tensor(np.asarray(wQ, float))
    wt = torch.as_tensor(np.asarray(wTw, float))
    s = (wq[usable] * Q[usable]).sum() + (wt[good] * Tw[good]).sum()
    s.backward()
    return Bt.grad.numpy(), log


def vjp_sample(B, grid, origin, u, v, nu, nv, seeds, wQ, wTw, p=None):
    """J^T w for weights on a sample of seeds only (wQ, wTw: one per sample
    seed): traces just the sample's lines and their lattice neighbours, so it
    scales to full-size lattices. Same masks as vjp()."""
    p = p or params()
    B = _f64(B)
    seeds = np.asarray(seeds, dtype=np.int64)
    lines = neighbourhood(seeds, nu, nv)
    log = lattice_log(B, grid, origin, u, v, nu, nv, p, which=lines)
    Bt = torch.tensor(B, dtype=torch.float64, requires_grad=True)
    Q, Tw, usable, _ = qmap_t(Bt, grid, origin, u, v, nu, nv, log, lines=lines, targets=seeds)
    row = {int(l): k for k, l in enumerate(lines)}
    good = torch.from_numpy((log["status"][[row[int(s)] for s in seeds]] & BAD) == 0)
    wq = torch.as_tensor(np.asarray(wQ, float))
    wt = torch.as_tensor(np.asarray(wTw, float))
    s = (wq[usable] * Q[usable]).sum() + (wt[good] * Tw[good]).sum()
    s.backward()
    return Bt.grad.numpy(), dict(Q=Q.detach().numpy(), Tw=Tw.detach().numpy(), usable=usable.numpy(),
                                 good=good.numpy(), lines=lines)


def jvp(B, grid, origin, u, v, nu, nv, dB, p=None, log=None):
    """Tangent-linear mode J v: the directional derivatives (dQ, dTw) of the
    frozen-sequence map along dB (forward-mode AD), and the usable mask."""
    import torch.autograd.forward_ad as fwAD

    p = p or params()
    B = _f64(B)
    log = lattice_log(B, grid, origin, u, v, nu, nv, p) if log is None else log
    with fwAD.dual_level():
        Bt = fwAD.make_dual(torch.tensor(B, dtype=torch.float64), torch.tensor(_f64(dB)))
        Q, Tw, usable, _ = qmap_t(Bt, grid, origin, u, v, nu, nv, log)
        dQ = fwAD.unpack_dual(Q).tangent
        dTw = fwAD.unpack_dual(Tw).tangent
        out = (dQ.numpy().copy(), dTw.numpy().copy(), usable.numpy())
    return out + (log,)


def free_loss(B, grid, origin, u, v, nu, nv, Qt, Twt, use, p=None, wtw=0.1):
    """The same loss from a free re-trace with the C oracle (step sizes chosen
    afresh), over a fixed seed mask: for finite differences of the true map."""
    p = p or params()
    o = plane(B, grid, origin, u, v, nu, nv, p)
    q, tw = o["Q"][use], o["Tw"][use]
    lq = np.log10(q) - np.log10(np.asarray(Qt)[use])
    return float(np.sum(lq * lq + wtw * (tw - np.asarray(Twt)[use]) ** 2) / max(int(use.sum()), 1))
