"""Seeded synthetic magnetic-field cubes.

Layout of every cube returned here: a C-contiguous array of shape
(nz, ny, nx, 3) (x fastest, the three Cartesian components innermost),
sampled at the nodes x_i = origin_x + i * spacing_x (and likewise for y, z),
or at the node coordinates of a stretched RectGrid.

Workloads (stand-ins for the paper's active-region extrapolation and TD99
runs, whose data are not available):

* analytic fields on [-1,1]^2 x [0,1] with 64^3 nodes (hyperbolic, rigid
  rotation, uniform, closed loops);
* potential fields of buried point monopoles, B = sum_i q_i (r - r_i)/|r - r_i|^3
  (the same form as the paper's quadrupole test field, Sec. 3.2), with seeded
  strengths, positions and depths;
* the paper's own quadrupole (Sec. 3.2, Eq. quadrapole) on a 0.02 grid;
* a rigid-twist flux tube superposed on a monopole cube (differentiation case).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Grid:
    """Uniform Cartesian grid: node counts, physical origin and spacing per axis."""

    n: tuple  # (nx, ny, nz)
    origin: tuple  # (x0, y0, z0)
    spacing: tuple  # (dx, dy, dz)

    @property
    def shape(self):
        nx, ny, nz = self.n
        return (nz, ny, nx, 3)

    @property
    def hi(self):
        return tuple(o + d * (k - 1) for o, d, k in zip(self.origin, self.spacing, self.n))

    def axis(self, a):
        return self.origin[a] + self.spacing[a] * np.arange(self.n[a], dtype=np.float64)


@dataclass(frozen=True)
class RectGrid:
    """Stretched (rectilinear) grid: strictly increasing node coordinates per
    axis, ``coords`` = (x, y, z) as tuples of floats."""

    coords: tuple

    @property
    def n(self):
        return tuple(len(c) for c in self.coords)

    @property
    def shape(self):
        nx, ny, nz = self.n
        return (nz, ny, nx, 3)

    @property
    def origin(self):
        return tuple(float(c[0]) for c in self.coords)

    @property
    def hi(self):
        return tuple(float(c[-1]) for c in self.coords)

    def axis(self, a):
        return np.asarray(self.coords[a], dtype=np.float64)


def stretched_axis(n: int, lo: float, hi: float, ratio: float, kind: str = "bottom"):
    """n node coordinates from lo to hi whose cell widths grow geometrically by
    ``ratio`` per cell: from the low end ('bottom') or from the middle towards
    both ends ('edges'). ratio = 1 gives the uniform axis."""
    m = n - 1
    if kind == "bottom":
        e = np.arange(m, dtype=np.float64)
    elif kind == "edges":
        e = np.abs(np.arange(m, dtype=np.float64) - 0.5 * (m - 1))
    else:
        raise ValueError(kind)
    w = ratio ** e
    x = np.concatenate([[0.0], np.cumsum(w)])
    x = lo + (hi - lo) * x / x[-1]
    x[0], x[-1] = lo, hi
    return tuple(float(v) for v in x)


def stretched_grid(n, lo, hi, ratios=(1.01, 1.01, 1.02), kinds=("edges", "edges", "bottom")):
    """RectGrid over the box [lo, hi] with the axes of stretched_axis."""
    return RectGrid(tuple(stretched_axis(int(n[a]), float(lo[a]), float(hi[a]), ratios[a], kinds[a])
                          for a in range(3)))


def _grid_from_box(n, lo, hi):
    sp = tuple((h - l) / (k - 1) for l, h, k in zip(lo, hi, n))
    return Grid(tuple(int(k) for k in n), tuple(float(v) for v in lo), sp)


ANALYTIC_GRID = _grid_from_box((64, 64, 64), (-1.0, -1.0, 0.0), (1.0, 1.0, 1.0))


def analytic_cube(kind: str, grid: Grid = ANALYTIC_GRID, q: float = 2.0 * math.pi,
                  dtype=np.float64):
    """Sample an analytic field at the nodes of ``grid``.

    kind: 'hyperbolic' B=(x,-y,1); 'rotation' B=(-q y, q x, 1);
    'uniform' B=(0,0,1); 'loops' B=(-y, x, 0) (closed circles, never exit);
    'null' B=(x, y, -2z) (a 3D null at the origin); 'expanding'
    B=(x/2, 0, 1-z/2); 'shear' B=(y/2, 0, 1); 'tilted' B=(1, 0, 0.02);
    'zero' B=0; 'linear' a generic traceless affine field. All are divergence-free and linear, so trilinear
    interpolation reproduces them exactly.
    """
    x, y, z = (grid.axis(a) for a in range(3))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    one = np.ones_like(X)
    if kind == "hyperbolic":
        B = (X, -Y, one)
    elif kind == "rotation":
        B = (-q * Y, q * X, one)
    elif kind == "uniform":
        B = (0 * X, 0 * X, one)
    elif kind == "loops":
        B = (-Y, X, 0 * X)
    elif kind == "null":
        B = (X, Y, -2.0 * Z)
    elif kind == "expanding":
        B = (0.5 * X, 0 * X, 1.0 - 0.5 * Z)
    elif kind == "shear":
        B = (0.5 * Y, 0 * X, one)
    elif kind == "tilted":
        B = (one, 0 * X, 0.02 * one)
    elif kind == "zero":
        B = (0 * X, 0 * X, 0 * X)
    elif kind == "linear":
        # a generic traceless (divergence-free) affine field with Bz > 0.3 in the box
        B = (0.6 * X - 0.5 * Y + 0.1 * Z + 0.05, 0.4 * X - 0.2 * Y - 0.1 + 0 * Z,
             0.2 * X + 0.1 * Y - 0.4 * Z + 1.0)
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(np.stack(B, axis=-1).astype(dtype))


def random_charges(rng: np.random.Generator, count: int, footprint, depth=(4.0, 16.0)):
    """Signed point-monopole sources below z=0.

    Strengths ~ N(0,1) rebalanced to zero net flux; horizontal positions uniform
    over ``footprint`` = ((x0, x1), (y0, y1)); depths uniform in ``depth``.
    Returns an array (count, 4) of (x, y, z, q).
    """
    q = rng.standard_normal(count)
    q -= q.mean()
    (x0, x1), (y0, y1) = footprint
    x = rng.uniform(x0, x1, count)
    y = rng.uniform(y0, y1, count)
    z = -rng.uniform(depth[0], depth[1], count)
    return np.stack([x, y, z, q], axis=1)


def perturbed_charges(charges, rng: np.random.Generator, rel=0.05):
    """Same sources with strengths scaled by (1 + rel * N(0,1))."""
    c = np.array(charges, dtype=np.float64, copy=True)
    c[:, 3] *= 1.0 + rel * rng.standard_normal(len(c))
    return c


def monopole_cube(grid: Grid, charges, dtype=np.float32, device=None):
    """B = sum_i q_i (r - r_i) / |r - r_i|^3 sampled at the grid nodes.

    Accumulated in float64, then rounded to ``dtype``. With ``device`` set
    (a torch device string) the sampling runs in torch on that device and a
    torch tensor is returned; otherwise a numpy array.
    """
    charges = np.asarray(charges, dtype=np.float64)
    nx, ny, nz = grid.n
    if device is not None:
        import torch

        tdt = {np.float32: torch.float32, np.float64: torch.float64}[np.dtype(dtype).type]
        out = torch.empty((nz, ny, nx, 3), dtype=tdt, device=device)
        xs = torch.tensor(grid.axis(0), dtype=torch.float64, device=device)
        ys = torch.tensor(grid.axis(1), dtype=torch.float64, device=device)
        zs = grid.axis(2)
        for k in range(nz):
            Y, X = torch.meshgrid(ys, xs, indexing="ij")
            acc = torch.zeros((ny, nx, 3), dtype=torch.float64, device=device)
            for cx, cy, cz, cq in charges:
                dx = X - cx
                dy = Y - cy
                dz = torch.full_like(X, zs[k] - cz)
                r2 = dx * dx + dy * dy + dz * dz
                s = cq / (r2 * torch.sqrt(r2))
                acc[..., 0] += s * dx
                acc[..., 1] += s * dy
                acc[..., 2] += s * dz
            out[k] = acc.to(tdt)
        return out
    out = np.empty((nz, ny, nx, 3), dtype=dtype)
    x = grid.axis(0)
    y = grid.axis(1)
    Y, X = np.meshgrid(y, x, indexing="ij")
    for k, zk in enumerate(grid.axis(2)):
        acc = np.zeros((ny, nx, 3), dtype=np.float64)
        for cx, cy, cz, cq in charges:
            dx = X - cx
            dy = Y - cy
            dz = zk - cz
            r2 = dx * dx + dy * dy + dz * dz
            s = cq / (r2 * np.sqrt(r2))
            acc[..., 0] += s * dx
            acc[..., 1] += s * dy
            acc[..., 2] += s * dz
        out[k] = acc.astype(dtype)
    return out


def monopole24_stretched(seed: int = 2208, n=(256, 256, 128), count: int = 24, dtype=np.float32,
                 ratios=(1.01, 1.01, 1.02)):
    """The 24-monopole field of monopole24_cube (same sources) sampled on a
    stretched grid over the same box: horizontal cells growing by ratios[0],
    ratios[1] per cell from the middle to the edges, vertical cells by
    ratios[2] per cell upward. Returns (B, RectGrid, charges)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    ch = random_charges(rng, count, ((0.0, nx - 1.0), (0.0, ny - 1.0)))
    grid = stretched_grid(n, (0.0, 0.0, 0.0), (nx - 1.0, ny - 1.0, nz - 1.0), ratios)
    return monopole_cube(grid, ch, dtype=dtype), grid, ch


def monopole24_cube(seed: int = 2208, n=(256, 256, 128), count: int = 24, dtype=np.float32,
                device=None):
    """Synthetic active-region potential field: ``count`` buried monopoles,
    unit spacing, origin 0, depths 4..16 cells. Returns (B, grid, charges)."""
    grid = Grid(tuple(n), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    rng = np.random.default_rng(seed)
    ch = random_charges(rng, count, ((0.0, n[0] - 1.0), (0.0, n[1] - 1.0)))
    return monopole_cube(grid, ch, dtype=dtype, device=device), grid, ch


def large_monopole(seed: int = 2208, n=(1024, 1024, 512), count: int = 64, device=None):
    """The large-volume workload: ``count`` buried monopoles (depths 4..16
    cells) on an FP32 cube of ``n`` nodes with unit spacing. Sampled on
    ``device`` (torch) when given. Returns (B, grid, charges)."""
    grid = Grid(tuple(n), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    rng = np.random.default_rng(seed)
    ch = random_charges(rng, count, ((0.0, n[0] - 1.0), (0.0, n[1] - 1.0)))
    return monopole_cube(grid, ch, dtype=np.float32, device=device), grid, ch


def quadrupole_charges():
    """The four unit charges of the paper's quadrupole (Sec. 3.2, Eq. quadrapole):
    +1, -1, +1, -1 at x = -1.5, -0.5, 0.5, 1.5, y = 0, z = -0.5."""
    return np.array([[-1.5, 0.0, -0.5, 1.0], [-0.5, 0.0, -0.5, -1.0],
                     [0.5, 0.0, -0.5, 1.0], [1.5, 0.0, -0.5, -1.0]])


def quadrupole_cube(spacing=0.02, box=((-3.0, 3.0), (-1.5, 1.5), (0.0, 1.5)),
                    dtype=np.float64):
    """The quadrupole sampled on a uniform grid of the given spacing (Sec. 3.2
    gives the spacing 0.02; the domain is not stated and is a reading)."""
    n = tuple(int(round((b[1] - b[0]) / spacing)) + 1 for b in box)
    grid = Grid(n, tuple(b[0] for b in box), (spacing,) * 3)
    return monopole_cube(grid, quadrupole_charges(), dtype=dtype), grid


def twist_tube_cube(grid: Grid, charges, turns: float = 1.5, radius_cells: float = 10.0,
                    dtype=np.float32):
    """Monopole potential field plus a vertical rigid-twist flux tube through
    the box centre: B_t = b0 w(r) (-q y', q x', 1) with w = exp(-r^2/R^2),
    q = 2 pi turns / H (H the box height), R = radius_cells * dx, and b0 the
    rms |B| of the potential field on z=0. div B_t = 0 for any radial w."""
    Bp = monopole_cube(grid, charges, dtype=np.float64)
    b0 = float(np.sqrt(np.mean(np.sum(Bp[0] ** 2, axis=-1))))
    x, y, z = (grid.axis(a) for a in range(3))
    xc = 0.5 * (x[0] + x[-1])
    yc = 0.5 * (y[0] + y[-1])
    H = z[-1] - z[0]
    q = 2.0 * math.pi * turns / H
    # a stretched grid has no spacing: its mean x width stands in
    dx = grid.spacing[0] if hasattr(grid, "spacing") else (x[-1] - x[0]) / (len(x) - 1)
    R = radius_cells * dx
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    xp = X - xc
    yp = Y - yc
    w = b0 * np.exp(-(xp * xp + yp * yp) / (R * R))
    Bp[..., 0] += -q * yp * w
    Bp[..., 1] += q * xp * w
    Bp[..., 2] += w
    return np.ascontiguousarray(Bp.astype(dtype)), dict(q=q, R=R, b0=b0, xc=xc, yc=yc)


def random_smooth_cube(rng: np.random.Generator, n=(8, 8, 8), lo=(0.0, 0.0, 0.0),
                       hi=(1.0, 1.0, 1.0), dtype=np.float64):
    """A small smooth random field: a uniform vertical component plus a few
    random monopoles placed well outside the box (no nulls inside)."""
    grid = _grid_from_box(n, lo, hi)
    ch = np.zeros((4, 4))
    ch[:, 0] = rng.uniform(lo[0], hi[0], 4)
    ch[:, 1] = rng.uniform(lo[1], hi[1], 4)
    ch[:, 2] = lo[2] - rng.uniform(0.5, 1.0, 4)
    ch[:, 3] = rng.uniform(-0.3, 0.3, 4)
    B = monopole_cube(grid, ch, dtype=np.float64)
    B[..., 2] += 1.0
    B[..., 0] += rng.uniform(-0.3, 0.3)
    B[..., 1] += rng.uniform(-0.3, 0.3)
    return np.ascontiguousarray(B.astype(dtype)), grid


BATCH_SIZES = ((64, 64, 64), (128, 128, 64), (256, 256, 128), (384, 384, 192))


def batch_specs(seed: int = 2208, count: int = 48, seeds_uv=(512, 256)):
    """Uneven batch: ``count`` monopole cubes of sizes drawn from BATCH_SIZES,
    8..64 sources each, each with either the z=0 plane or the vertical xz
    slice at mid-y as its seed plane (seeds_uv seeds, cell-centred)."""
    rng = np.random.default_rng(seed)
    specs = []
    for b in range(count):
        n = BATCH_SIZES[int(rng.integers(len(BATCH_SIZES)))]
        ncharge = int(rng.integers(8, 65))
        depth = (4.0 * n[0] / 256.0 + 1.0, 16.0 * n[0] / 256.0 + 1.0)
        ch = random_charges(rng, ncharge, ((0.0, n[0] - 1.0), (0.0, n[1] - 1.0)), depth)
        grid = Grid(n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
        nu, nv = seeds_uv
        if rng.random() < 0.5:
            plane = dict(origin=(0.0, 0.0, 0.0), u=((n[0] - 1.0) / nu, 0.0, 0.0),
                         v=(0.0, (n[1] - 1.0) / nv, 0.0), nu=nu, nv=nv)
        else:
            plane = dict(origin=(0.0, (n[1] - 1.0) / 2.0, 0.0), u=((n[0] - 1.0) / nu, 0.0, 0.0),
                         v=(0.0, 0.0, (n[2] - 1.0) / nv), nu=nu, nv=nv)
        specs.append(dict(grid=grid, charges=ch, plane=plane))
    return specs


def adjoint_cubes(seed: int = 2208, n=(128, 128, 64), count: int = 24, turns: float = 1.5,
                  radius_cells: float = 10.0, rel: float = 0.05, dtype=np.float32, ratios=None):
    """The differentiation workload: a monopole potential field (``count``
    buried sources, depths 4..16 cells scaled by nx/128, unit spacing) plus a
    vertical rigid-twist tube (``turns`` over the box height, radius
    ``radius_cells``), and the target cube: the same sources with strengths
    scaled by (1 + rel N(0,1)) under the same tube. With ``ratios`` the same
    sources are sampled on a stretched grid over the same box (stretched_grid's
    axes: horizontal widths growing by ratios[0], ratios[1] per cell from the
    middle, vertical by ratios[2] upward). Returns (B, B_target, grid)."""
    grid = Grid(tuple(n), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    if ratios is not None:
        grid = stretched_grid(n, (0.0, 0.0, 0.0), tuple(float(k - 1) for k in n), ratios)
    rng = np.random.default_rng(seed)
    s = n[0] / 128.0
    ch = random_charges(rng, count, ((0.0, n[0] - 1.0), (0.0, n[1] - 1.0)), depth=(4.0 * s, 16.0 * s))
    cht = perturbed_charges(ch, rng, rel)
    B, _ = twist_tube_cube(grid, ch, turns=turns, radius_cells=radius_cells, dtype=dtype)
    Bt, _ = twist_tube_cube(grid, cht, turns=turns, radius_cells=radius_cells, dtype=dtype)
    return B, Bt, grid
