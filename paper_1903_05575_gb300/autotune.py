"""Autotuner for the grouped path's tile shapes.

The paper picks its cache-blocking parameters per machine by black-box
search (Sec. 3.2; OpenTuner in Sec. 5).  The GPU analogue here is the tile
shape of each problem in a grouped batch: for each size bucket (the range of
m times the range of n, 25 buckets), every tile shape the library offers is
timed on a seeded synthetic batch of problems from that bucket, and the
fastest is kept.  FP64 batches choose among four DMMA tile shapes; split-BF16
batches among column-tile widths of 64, 32 and 16 quaternion columns (the
tcgen05 MMA width follows), by coordinate descent over the buckets on one
mixed batch, since a width that speeds up a bucket's own small batch can
slow a full one.  The tables are installed in the library
(qgemm_grouped_set_tile_table) and stored as JSON keyed by the GPU's name, its
SM count and the library version; a stored plan is applied only when the key
matches the current device.

  python -m paper_1903_05575_gb300.autotune [--out PATH] [--per-bucket N]
"""
import json
import os

import numpy as np

from . import _abi, ops

RANGES = [(1, 16), (17, 32), (33, 64), (65, 128), (129, 256)]
PLAN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plans")
_loaded = False


def device_key(device=0):
    import torch
    props = torch.cuda.get_device_properties(device)
    return {"gpu": props.name, "sms": props.multi_processor_count,
            "library": _abi.lib().qgemm_version().decode()}


def default_plan_path(key):
    env = os.environ.get("QGEMM_PLAN_CACHE")
    if env:
        return env
    name = "%s_%dsm.json" % (key["gpu"].replace(" ", "_"), key["sms"])
    return os.path.join(PLAN_DIR, name)


def bucket_problems(rm, rn, count, seed, kmax=256):
    """Sizes and ops of a synthetic batch in bucket (rm, rn)."""
    g = np.random.Generator(np.random.PCG64(seed))
    lo_m, hi_m = RANGES[rm]
    lo_n, hi_n = RANGES[rn]
    out = []
    for _ in range(count):
        out.append(dict(m=int(g.integers(lo_m, hi_m + 1)), n=int(g.integers(lo_n, hi_n + 1)),
                        k=int(g.integers(8, kmax + 1)),
                        opA="NH"[int(g.integers(0, 2))], opB="NH"[int(g.integers(0, 2))]))
    return out


def _time_batch(problems, reps):
    import torch
    b = ops.GroupedBatch(problems)
    b.launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        b.launch()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_grouped(per_bucket=96, reps=3, seed=2019, verbose=False):
    """Times every shape in every bucket (FP64 path); returns (table, report)
    and installs the table."""
    import torch
    global _loaded
    _loaded = True  # a stored plan must not replace the tables being timed
    shapes, nbuckets, _ = ops.tile_info()
    dev = torch.device("cuda", torch.cuda.current_device())
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    table, report = [], []
    for rm in range(len(RANGES)):
        for rn in range(len(RANGES)):
            specs = bucket_problems(rm, rn, per_bucket, seed + 31 * rm + rn)
            probs, flops = [], 0.0
            for p in specs:
                ra, ca = (p["k"], p["m"]) if p["opA"] == "H" else (p["m"], p["k"])
                rb, cb = (p["n"], p["k"]) if p["opB"] == "H" else (p["k"], p["n"])
                probs.append(dict(p, alpha=(1.0, 0, 0, 0), beta=(0.0, 0, 0, 0),
                                  A=torch.randn((ca, ra, 4), dtype=torch.float64, device=dev,
                                                generator=gen),
                                  B=torch.randn((cb, rb, 4), dtype=torch.float64, device=dev,
                                                generator=gen),
                                  C=torch.empty((p["n"], p["m"], 4), dtype=torch.float64,
                                                device=dev)))
                flops += 32.0 * p["m"] * p["n"] * p["k"]
            times = []
            for s in range(len(shapes)):
                ops.set_tile_table([s] * nbuckets)
                times.append(_time_batch(probs, reps))
            best = int(np.argmin(times))
            table.append(best)
            rec = {"bucket": [rm, rn], "m_range": RANGES[rm], "n_range": RANGES[rn],
                   "ms": times, "tflops": [flops / (t * 1e-3) / 1e12 for t in times],
                   "best": best, "best_shape": shapes[best]}
            report.append(rec)
            if verbose:
                print(json.dumps(rec), flush=True)
    ops.set_tile_table(table)
    return table, report


SPLIT_WIDTHS = [64, 32, 16]   # column-tile width of code 0, 1, 2


def mixed_problems(count, seed, kmax=256):
    """Sizes and ops of a mixed batch: m, n, k uniform in [8, kmax], ops in {N, H}."""
    g = np.random.Generator(np.random.PCG64(seed))
    return [dict(m=int(g.integers(8, kmax + 1)), n=int(g.integers(8, kmax + 1)),
                 k=int(g.integers(8, kmax + 1)), opA="NH"[int(g.integers(0, 2))],
                 opB="NH"[int(g.integers(0, 2))]) for _ in range(count)]


def tune_grouped_split(count=1024, reps=10, seed=2029, gain=0.01, verbose=False):
    """Column-tile widths of split-BF16 batches by coordinate descent on a
    seeded mixed batch (FP32, unit-quaternion alpha and beta): starting from
    width 64 everywhere, each bucket in turn takes the width that makes the
    whole batch fastest, if it gains more than `gain` (a width that helps a
    bucket alone can slow a full batch, whose per-tile costs dominate).
    Returns (table, report) and installs the table."""
    import torch
    global _loaded
    _loaded = True
    rng = np.random.Generator(np.random.PCG64(seed))

    def unit():
        q = rng.standard_normal(4)
        return tuple(float(x) for x in q / np.linalg.norm(q))
    dev = torch.device("cuda", torch.cuda.current_device())
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    probs, flops = [], 0.0
    for p in mixed_problems(count, seed):
        ra, ca = (p["k"], p["m"]) if p["opA"] == "H" else (p["m"], p["k"])
        rb, cb = (p["n"], p["k"]) if p["opB"] == "H" else (p["k"], p["n"])
        probs.append(dict(p, alpha=unit(), beta=unit(),
                          A=torch.randn((ca, ra, 4), dtype=torch.float32, device=dev,
                                        generator=gen),
                          B=torch.randn((cb, rb, 4), dtype=torch.float32, device=dev,
                                        generator=gen),
                          C=torch.randn((p["n"], p["m"], 4), dtype=torch.float32, device=dev,
                                        generator=gen)))
        flops += 32.0 * p["m"] * p["n"] * p["k"]

    def timed(tbl):
        ops.set_tile_table(tbl, precision="split_bf16")
        return _time_batch(probs, reps)
    table = [0] * 25
    best = timed(table)
    report = [{"start_ms": best, "tflops": flops / (best * 1e-3) / 1e12}]
    for bkt in range(25):
        trial = {}
        for code in range(1, len(SPLIT_WIDTHS)):
            t = list(table)
            t[bkt] = code
            trial[code] = timed(t)
        code = min(trial, key=trial.get)
        if trial[code] < best * (1.0 - gain):
            table[bkt] = code
            best = trial[code]
        rec = {"bucket": [bkt // 5, bkt % 5], "ms": [trial.get(c) for c in range(1, 3)],
               "kept": SPLIT_WIDTHS[table[bkt]], "batch_ms": best}
        report.append(rec)
        if verbose:
            print(json.dumps(rec), flush=True)
    report.append({"final_ms": best, "tflops": flops / (best * 1e-3) / 1e12})
    ops.set_tile_table(table, precision="split_bf16")
    return table, report


def save_plan(table, report, path=None, split_table=None, split_report=None):
    key = device_key()
    path = path or default_plan_path(key)
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    shapes, nbuckets, edges = ops.tile_info()
    plan = {"key": key, "precision": "fp64", "shapes": shapes, "edges": edges,
            "table": table, "report": report}
    if split_table is not None:
        plan.update({"split_widths": SPLIT_WIDTHS, "split_table": split_table,
                     "split_report": split_report})
    with open(path, "w") as f:
        json.dump(plan, f, indent=1)
    return path


def plan_matches(plan, key):
    return (isinstance(plan, dict) and plan.get("key") == key and plan.get("precision") == "fp64"
            and isinstance(plan.get("table"), list) and len(plan["table"]) == 25)


def load_plan(path=None, key=None, install=True):
    """Applies a stored plan if it exists and matches the device; returns the
    table or None."""
    key = key or device_key()
    path = path or default_plan_path(key)
    try:
        with open(path) as f:
            plan = json.load(f)
    except (OSError, ValueError):
        return None
    if not plan_matches(plan, key):
        return None
    if install:
        ops.set_tile_table(plan["table"])
        st = plan.get("split_table")
        if isinstance(st, list) and len(st) == 25:
            ops.set_tile_table(st, precision="split_bf16")
    return plan["table"]


def ensure_plan_loaded():
    """Once per process: apply the stored plan for this device if there is one."""
    global _loaded
    if not _loaded:
        _loaded = True
        try:
            load_plan()
        except Exception:  # no device or no plan: the library's default table stays
            pass


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--per-bucket", type=int, default=96)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--split-only", action="store_true",
                    help="keep the stored FP64 table, tune the split-BF16 widths")
    a = ap.parse_args()
    if a.split_only:
        key = device_key()
        with open(a.out or default_plan_path(key)) as f:
            old = json.load(f)
        tbl, rep = old["table"], old.get("report")
    else:
        tbl, rep = tune_grouped(per_bucket=a.per_bucket, reps=a.reps, verbose=True)
    stbl, srep = tune_grouped_split(verbose=True)
    print("fp64 table", tbl)
    print("split table", stbl)
    print("saved", save_plan(tbl, rep, a.out, stbl, srep))
