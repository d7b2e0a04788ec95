"""Host logic of the scheduling autotuner (CPU): an exhaustive search over the
knob space that keeps the fastest setting, a per-(GPU, workload) JSON cache
that a later call reuses without timing, and force / no-cache modes. Timing
and the device name are replaced by fakes; nothing runs on a GPU."""
import json

import pytest

pytest.importorskip("torch")


@pytest.fixture()
def at(monkeypatch):
    try:
        from paper_2208_12569_gb300 import autotune
    except (ImportError, OSError) as e:  # the library is built by __graft_entry__.build()
        pytest.skip("libfqsl.so not built: %s" % e)
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda *a: "FAKE GPU")
    return autotune


def _fake(at, monkeypatch, calls):
    # time = a made-up function of the knobs, minimal at refill 16, sync 1,
    # chunk 4, blocks 2
    def cost(p):
        return (abs(p.refill_lanes - 16) + 3 * abs(p.sync_dirs - 1) + abs(p.chunk_tiles - 4)
                + 2 * abs(p.blocks_per_sm - 2) + 1.0)

    current = {}

    def run_with(p):
        calls.append((p.refill_lanes, p.sync_dirs, p.chunk_tiles, p.blocks_per_sm))
        current["p"] = p

    monkeypatch.setattr(at, "_time", lambda run, reps: (run(), cost(current["p"]))[1])
    return run_with


def test_search_cache_and_force(at, monkeypatch, tmp_path):
    from paper_2208_12569_gb300 import fqsl

    path = str(tmp_path / "tune.json")
    calls = []
    run_with = _fake(at, monkeypatch, calls)
    base = fqsl.params(tol=1e-4)
    best, table = at.tune(run_with, base, key="w1", path=path, warmup=1)
    space = at.DEFAULT_SPACE
    n = 1
    for v in space.values():
        n *= len(v)
    assert len(table) == n
    assert (best.refill_lanes, best.sync_dirs, best.chunk_tiles, best.blocks_per_sm) == (16, 1, 4, 2)
    assert best.tol == 1e-4  # the non-scheduling fields are the caller's
    assert min(r["ms"] for r in table) == 1.0
    assert len(calls) == 2 * n  # one warm-up and one timed run per setting
    data = json.load(open(path))
    assert "FAKE GPU|w1" in data and data["FAKE GPU|w1"]["best"]["refill_lanes"] == 16
    # a second call reads the cache and runs nothing
    calls.clear()
    best2, _ = at.tune(run_with, fqsl.params(tol=2e-4), key="w1", path=path)
    assert calls == [] and best2.refill_lanes == 16 and best2.tol == 2e-4
    # another workload key is tuned afresh and kept beside the first
    at.tune(run_with, base, key="w2", path=path, space={"refill_lanes": (1, 32)})
    data = json.load(open(path))
    assert set(data) == {"FAKE GPU|w1", "FAKE GPU|w2"}
    assert data["FAKE GPU|w2"]["best"] == {"refill_lanes": 1}  # |1 - 16| < |32 - 16|
    # force re-times despite the cache; path '' keeps no cache
    calls.clear()
    at.tune(run_with, base, key="w1", path=path, force=True, space={"sync_dirs": (0, 1)}, warmup=0)
    assert len(calls) == 2
    calls.clear()
    at.tune(run_with, base, key="w3", path="", space={"sync_dirs": (0, 1)}, warmup=0)
    assert len(calls) == 2 and "FAKE GPU|w3" not in json.load(open(path))
