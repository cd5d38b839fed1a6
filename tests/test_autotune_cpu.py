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


def test_split_width_table_sets_the_tile_count():
    """Split-BF16 batches: the per-bucket column-tile width (codes 0, 1, 2 for
    64, 32, 16 columns) is installed by qgemm_grouped_set_tile_table and
    decides how many tiles (16-byte entries) a problem's schedule has."""
    import ctypes

    from paper_1903_05575_gb300 import _abi
    L = _abi.lib()
    count = 32
    arr = (_abi.QgemmProblem * count)()
    for q in arr:
        q.opA = q.opB = 0
        q.m, q.n, q.k = 100, 200, 40   # bucket (65-128, 129-256), computed as it is
        q.alpha[0] = 1.0
        q.A = q.B = q.C = 64
        q.lda, q.ldb, q.ldc = 100, 40, 100

    def ws_with(code):
        tbl = (ctypes.c_int32 * 25)(*([code] * 25))
        assert L.qgemm_grouped_set_tile_table(_abi.PRECISION["split_bf16"], tbl, 25) == 0
        return L.qgemm_grouped_workspace_bytes(arr, count, 0, _abi.PRECISION["split_bf16"])
    try:
        sizes = [ws_with(c) for c in range(3)]
        bad = (ctypes.c_int32 * 25)(*([3] * 25))
        assert L.qgemm_grouped_set_tile_table(_abi.PRECISION["split_bf16"], bad, 25) == -2
    finally:
        assert L.qgemm_grouped_set_tile_table(_abi.PRECISION["split_bf16"], None, 0) == 0
    # 1 row tile x ceil(200 / w) column tiles, 16 bytes each (up to 256-byte rounding)
    tiles = [-(-200 // w) for w in autotune.SPLIT_WIDTHS]
    assert tiles == [4, 7, 13]
    assert sizes[0] < sizes[1] < sizes[2]
    assert abs((sizes[2] - sizes[0]) - 16 * count * (tiles[2] - tiles[0])) <= 512
