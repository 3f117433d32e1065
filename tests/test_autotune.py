"""Autotuner host logic (no GPU): size buckets, the JSON cache, nearest-bucket
lookup, and the coordinate-descent search on a synthetic cost model."""
import json

import pytest

from paper_1205_6693_gb300 import autotune as A


def test_buckets():
    assert A.bucket(16_777_216) == "single:r24"
    assert A.bucket(12_000_000) == "single:r24"  # log2 = 23.5 rounds up
    assert A.bucket(11_000_000) == "single:r23"
    assert A.bucket(0) == "single:r0"
    assert A.bucket(38_700_000, 4096) == "batch:r25:g12"


def test_cache_roundtrip_and_lookup(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "schedules.json"
    monkeypatch.setenv("TRUSS_TUNE_CACHE", str(path))
    assert A.load() == {}
    key = "GB300|sm_103|152SM"
    cache = {key: {"single:r20": {"opts": {"peel_variant": 1}},
                   "single:r24": {"opts": {"peel_variant": 3}},
                   "batch:r25:g12": {"opts": {"support_range_work": 4096}}}}
    A.save(cache)
    assert json.loads(path.read_text()) == cache
    assert A.lookup(key, 1 << 20) == {"peel_variant": 1}
    assert A.lookup(key, 1 << 23) == {"peel_variant": 3}  # nearest single bucket
    assert A.lookup(key, 1 << 23, nearest=False) is None
    assert A.lookup(key, 1 << 25, 4000) == {"support_range_work": 4096}
    assert A.lookup(key, 1 << 10, 2) == {"support_range_work": 4096}  # only batch entry
    assert A.lookup("other gpu", 1 << 20) is None
    path.write_text("not json")
    assert A.load() == {}


def _cost_model(opts):
    # separable convex costs with a known optimum per knob
    best = {"support_range_work": 8192, "support_stage_max": 128, "support_pair_cost": 16,
            "peel_variant": 1}
    sup = 10.0
    for k in ("support_range_work", "support_stage_max", "support_pair_cost"):
        sup += 0.0 if opts.get(k, 0) == best[k] else 1.0
    peel = 5.0 if opts.get("peel_variant", 0) == best["peel_variant"] else 7.0
    return {"ms_support": sup, "ms_lists": 1.0, "ms_peel": peel}


def test_search_finds_the_separable_optimum():
    seen = []

    def run(opts):
        seen.append(opts)
        return _cost_model(opts), ("same",)

    opts, ms, calls = A.search(run, reps=2, same=lambda a, b: a == b)
    assert opts == {"support_range_work": 8192, "support_stage_max": 128,
                    "support_pair_cost": 16, "peel_variant": 1, "lists_in_place": 0}
    assert ms["ms_support"] == 10.0 and ms["ms_peel"] == 5.0
    distinct = 1 + sum(len(v) - 1 for v in A.SPACE.values())
    assert calls == 2 * distinct == len(seen)


def test_search_keeps_default_without_a_clear_gain():
    def run(opts):
        st = {"ms_support": 10.0, "ms_lists": 1.0, "ms_peel": 5.0}
        if opts.get("peel_variant") == 3:
            st["ms_peel"] = 4.95  # 1 % better: below min_gain
        return st, 0

    opts, _, _ = A.search(run, reps=1)
    assert all(v == 0 for v in opts.values())


def test_search_rejects_a_schedule_that_changes_results():
    def run(opts):
        return _cost_model(opts), (opts.get("support_stage_max", 0) == 64,)

    with pytest.raises(RuntimeError, match="changed the result"):
        A.search(run, reps=1, same=lambda a, b: a == b)
