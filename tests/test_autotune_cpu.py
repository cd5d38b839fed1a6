"""Host logic of the grouped-path autotuner (no GPU): bucket sampling and
plan keys."""
import json

from paper_1903_05575_gb300 import autotune, tile_info


def test_buckets_match_library_edges():
    shapes, nbuckets, edges = tile_info()
    assert nbuckets == len(autotune.RANGES) ** 2
    assert [hi for _, hi in autotune.RANGES[:-1]] == edges
    assert len(shapes) >= 2


def test_bucket_problems_stay_in_range_and_are_seeded():
    for rm in range(5):
        for rn in range(5):
            ps = autotune.bucket_problems(rm, rn, 50, seed=3)
            lo_m, hi_m = autotune.RANGES[rm]
            lo_n, hi_n = autotune.RANGES[rn]
            assert all(lo_m <= p["m"] <= hi_m and lo_n <= p["n"] <= hi_n and 8 <= p["k"] <= 256
                       for p in ps)
    assert autotune.bucket_problems(2, 3, 10, 5) == autotune.bucket_problems(2, 3, 10, 5)


def test_plan_applied_only_for_matching_key(tmp_path):
    key = {"gpu": "NVIDIA GB300", "sms": 152, "library": "x"}
    plan = {"key": key, "precision": "fp64", "table": [3] * 25}
    path = tmp_path / "plan.json"
    path.write_text(json.dumps(plan))
    assert autotune.load_plan(str(path), key=key, install=False) == [3] * 25
    other = dict(key, sms=148)
    assert autotune.load_plan(str(path), key=other, install=False) is None
    path.write_text(json.dumps(dict(plan, table=[1] * 24)))
    assert autotune.load_plan(str(path), key=key, install=False) is None
    assert autotune.load_plan(str(tmp_path / "missing.json"), key=key, install=False) is None
