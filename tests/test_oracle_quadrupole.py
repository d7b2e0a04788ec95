"""Paper's own worked case (Sec. 3.2, Eq. quadrapole; fixture in
tests/golden/quadrupole.json): in the regions whose lines cross the symmetry
plane x = 0 the footpoint map is x2 = -x1, y2 = y1 and Q = 2 exactly."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "quadrupole.json")))


@pytest.fixture(scope="module")
def quad():
    charges = np.array(GOLD["charges_xyzq"])
    assert np.array_equal(charges, synth.quadrupole_charges())
    B, grid = synth.quadrupole_cube(GOLD["grid_spacing"], tuple(map(tuple, GOLD["domain_reading"])))
    assert grid.n == (301, 151, 76)
    return B, grid, oracle.curl(B, grid)


@pytest.mark.parametrize("method,way", [(1, 1), (2, 2)])
def test_quadrupole_reflection_map_and_q2(oracle_lib, quad, method, way):
    B, grid, J = quad
    n = 16
    d = 0.0125
    # a patch in the "in" region between the inner spots (x = -0.5 and +0.5)
    o = oracle.plane(B, grid, (0.02, -0.1, 0.0), (d, 0, 0), (0, d, 0), n, n,
                     oracle.params(method=method, way=way, tol=1e-10), J=J)
    xs = 0.02 + (np.arange(n) + 0.5) * d
    ys = -0.1 + (np.arange(n) + 0.5) * d
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    X, Y = X.ravel(), Y.ravel()
    cross = (o["face2"] == 4) & (o["r2"][:, 0] < 0)
    assert cross.sum() == n * n
    assert np.max(np.abs(o["r2"][cross, 0] + X[cross])) < 1e-7
    assert np.max(np.abs(o["r2"][cross, 1] - Y[cross])) < 1e-7
    # Q = 2 where the seed and all four neighbours cross (FD of a reflection is exact)
    C = cross.reshape(n, n)
    inner = np.zeros_like(C)
    inner[1:-1, 1:-1] = C[1:-1, 1:-1] & C[2:, 1:-1] & C[:-2, 1:-1] & C[1:-1, 2:] & C[1:-1, :-2]
    inner = inner.ravel()
    assert inner.sum() > 10
    # Method I: footpoint errors ~1e-8 over the lattice step 0.0125 bound the FD
    # error; Method II way 2 carries the +-0.001-cell difference error of grad(B/B)
    tol = 2e-6 if method == 1 else 1e-3
    assert np.max(np.abs(o["Q"][inner] - GOLD["expected"]["Q_in_out_regions"])) < tol
