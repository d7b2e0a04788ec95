"""Brute-force pin of the oracle's tracer on tiny random grids: an independent
integration of the field-line equation (Sec. 2.1, Eq. rb) and the twist
integrand (Eq. tw) with scipy's DOP853 at tight tolerance, on scipy's own
trilinear interpolant of the same nodes (Sec. 2.2, Eq. interp) and numpy's
differences for the curl, with exact face crossings from event location."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.interpolate import RegularGridInterpolator

import oracle
import synth


def _scipy_trace(B, grid, seed, sign):
    axes = tuple(grid.axis(a) for a in range(3))
    comps = [RegularGridInterpolator(axes, np.transpose(B[..., m], (2, 1, 0))) for m in range(3)]
    dx, dy, dz = grid.spacing
    g = [np.gradient(B[..., m], dz, dy, dx, edge_order=2)[::-1] for m in range(3)]
    J = np.stack([g[2][1] - g[1][2], g[0][2] - g[2][0], g[1][0] - g[0][1]], -1)
    jc = [RegularGridInterpolator(axes, np.transpose(J[..., m], (2, 1, 0))) for m in range(3)]
    lo = np.array(grid.origin)
    hi = np.array(grid.hi)

    def rhs(s, y):
        r = np.clip(y[:3], lo, hi)[None]
        b = np.array([c(r)[0] for c in comps])
        j = np.array([c(r)[0] for c in jc])
        nb = np.linalg.norm(b)
        return np.concatenate([sign * b / nb, [1.0, j @ b / (4 * math.pi * nb * nb)]])

    events = []
    for a in range(3):
        for bound in (lo[a], hi[a]):
            ev = (lambda s, y, a=a, bound=bound: y[a] - bound)
            ev.terminal = True
            events.append(ev)
    y0 = np.concatenate([seed, [0.0, 0.0]])
    sol = solve_ivp(rhs, (0.0, 50.0), y0, method="DOP853", rtol=1e-13, atol=1e-13, events=events,
                    max_step=0.05)
    return sol.y[:, -1]


@pytest.mark.parametrize("seed_rng", [11, 12])
def test_tracer_matches_scipy_dop853(oracle_lib, seed_rng):
    rng = np.random.default_rng(seed_rng)
    B, grid = synth.random_smooth_cube(rng, n=(8, 8, 8))
    seeds = rng.uniform(0.15, 0.85, size=(6, 3))
    out = oracle.trace(B, grid, seeds, 1e-12, oracle.params(hmax=1.0))
    for s in range(len(seeds)):
        fwd = _scipy_trace(B, grid, seeds[s], +1.0)
        bwd = _scipy_trace(B, grid, seeds[s], -1.0)
        r2 = oracle.physical(grid, out["ends"][s, 1, :3])
        r1 = oracle.physical(grid, out["ends"][s, 0, :3])
        cell = min(grid.spacing)
        assert np.max(np.abs(r2 - fwd[:3])) < 1e-8 * cell
        assert np.max(np.abs(r1 - bwd[:3])) < 1e-8 * cell
        length = out["ends"][s, 0, 3] + out["ends"][s, 1, 3]
        tw = out["ends"][s, 0, 4] + out["ends"][s, 1, 4]
        assert abs(length - (fwd[3] + bwd[3])) < 1e-8 * cell
        assert abs(tw - (fwd[4] + bwd[4])) < 1e-9
