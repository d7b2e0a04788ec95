"""Comparison helpers for CUDA-vs-oracle parity tests (bars from the parity
metric: FP64 median relative Q and Tw error <= 1e-9, 99th percentile <= 1e-4
over points with Q < 1e6; Tw relative to max(|Tw|, 1e-3); faces and status
bit-exact)."""
import numpy as np


def to_np(out):
    return {k: (t.cpu().numpy() if hasattr(t, "cpu") else t) for k, t in out.items() if t is not None}


def q_rel(g, r):
    ok = np.isfinite(r["Q"]) & (r["Q"] < 1e6)
    return np.abs(g["Q"][ok] / r["Q"][ok] - 1)


def tw_rel(g, r):
    ok = np.isfinite(r["Tw"])
    return np.abs(g["Tw"][ok] - r["Tw"][ok]) / np.maximum(np.abs(r["Tw"][ok]), 1e-3)


def assert_exact_ints(g, r, keys=("face1", "face2", "status")):
    for k in keys:
        gg, rr = np.asarray(g[k]).astype(np.int64), np.asarray(r[k]).astype(np.int64)
        bad = np.nonzero(gg != rr)[0]
        assert bad.size == 0, "%s differs at %d of %d seeds, first %s: gpu %s oracle %s" % (
            k, bad.size, gg.size, bad[:5], gg[bad[:5]], rr[bad[:5]])


def assert_nan_pattern(g, r):
    for k in ("Q", "Tw", "length"):
        if k in g and k in r:
            assert np.array_equal(np.isnan(g[k]), np.isnan(r[k])), k


def assert_fp64_parity(g, r, med=1e-9, p99=1e-4):
    assert_exact_ints(g, r)
    assert_nan_pattern(g, r)
    if "Q" in r:
        rel = q_rel(g, r)
        if rel.size:
            assert np.median(rel) <= med and np.percentile(rel, 99) <= p99, (np.median(rel), np.percentile(rel, 99))
    t = tw_rel(g, r)
    if t.size:
        assert np.median(t) <= med and np.percentile(t, 99) <= p99, (np.median(t), np.percentile(t, 99))


def footpoint_cells_exact(g, r, grid, margin=1e-9):
    """Integer cell indices of the footpoints agree, except where the oracle's
    footpoint lies within ``margin`` cells of a cell boundary. Returns the
    number of excluded coordinates."""
    o = np.asarray(grid.origin)
    d = np.asarray(grid.spacing)
    ok = (r["status"] & 19) == 0
    excluded = 0
    for k in ("r1", "r2"):
        xr = (r[k][ok] - o) / d
        xg = (g[k][ok] - o) / d
        near = np.abs(xr - np.round(xr)) < margin
        excluded += int(near.sum())
        same = np.floor(xr) == np.floor(xg)
        assert np.all(same | near), "footpoint cell differs at %d coordinates" % int((~(same | near)).sum())
    return excluded


def assert_bitwise(g, r, keys=("Q", "Tw", "length", "r1", "r2", "face1", "face2", "status", "steps")):
    """Every output identical to the last bit (NaN where the oracle has NaN)."""
    for k in keys:
        if k not in r or k not in g:
            continue
        gg, rr = np.asarray(g[k]), np.asarray(r[k])
        if rr.dtype.kind == "f":
            same = (gg == rr) | (np.isnan(gg) & np.isnan(rr))
        else:
            same = gg.astype(np.int64) == rr.astype(np.int64)
        bad = np.nonzero(~same.reshape(len(rr), -1).all(axis=1))[0]
        assert bad.size == 0, "%s differs at %d of %d seeds, first %s: gpu %s oracle %s" % (
            k, bad.size, len(rr), bad[:3], gg[bad[:3]], rr[bad[:3]])
