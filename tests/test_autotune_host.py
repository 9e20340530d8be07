"""Host logic of the launch-shape autotuner's cache, on the CPU: shape
buckets, the nearest ensemble-size bucket, the operator form kept apart, and
the matrix-shape lookup with its default."""
import json

from paper_2603_03639_gb300 import autotune


def _cache(tmp_path, entries):
    p = tmp_path / "tuned.json"
    p.write_text(json.dumps(entries))
    return str(p)


def test_shape_buckets():
    # K, M*P and chi by powers of two; N and C exact; gradient and operator forms apart
    assert autotune.shape_key(50, 100, 64, 256, 8, 3) == "N50-C3-K128-T2048-chi64-grad"
    assert autotune.shape_key(50, 128, 33, 200, 8, 3) == "N50-C3-K128-T2048-chi64-grad"
    assert autotune.shape_key(50, 100, 20, 256, 1, 3, operator=True) == "N50-C3-K128-T256-chi32-grad-op"
    assert autotune.shape_key(50, 100, 64, 256, 8, 3, grad=False) == "N50-C3-K128-T2048-chi64-fid"
    assert autotune.shape_key(49, 100, 64, 256, 8, 3) != autotune.shape_key(50, 100, 64, 256, 8, 3)


def test_exact_and_nearest_ensemble_bucket(tmp_path):
    path = _cache(tmp_path, {
        "N50-C3-K128-T2048-chi64-grad": {"warps": 6, "ctas_per_sm": 1, "pairs": True},
        "N50-C3-K128-T64-chi64-grad": {"warps": 4, "ctas_per_sm": 2, "pairs": False},
    })
    assert autotune.lookup(50, 100, 64, 256, 8, 3, path=path) == (6, 1)
    assert autotune.lookup(50, 100, 64, 128, 8, 3, path=path) == (6, 1)     # T1024: nearest is T2048
    assert autotune.lookup(50, 100, 64, 8, 8, 3, path=path) == (4, 2)       # T64 exactly
    assert autotune.lookup(50, 100, 64, 2, 8, 3, path=path) == (4, 2)       # T16: nearest is T64
    # another K bucket, chi bucket or N has no entry: defaults
    assert autotune.lookup(50, 300, 64, 256, 8, 3, path=path) == (0, 0)
    assert autotune.lookup(50, 100, 16, 256, 8, 3, path=path) == (0, 0)
    assert autotune.lookup(30, 100, 64, 256, 8, 3, path=path) == (0, 0)


def test_operator_form_is_looked_up_apart(tmp_path):
    path = _cache(tmp_path, {
        "N50-C3-K128-T256-chi32-grad": {"warps": 8, "ctas_per_sm": 1, "pairs": True},
        "N50-C3-K128-T256-chi32-grad-op": {"warps": 4, "ctas_per_sm": 2, "pairs": False, "operator": True},
    })
    assert autotune.lookup(50, 100, 20, 256, 1, 3, path=path, operator=True) == (4, 2)
    assert autotune.lookup(50, 100, 20, 256, 1, 3, path=path) == (8, 1)
    assert autotune.lookup_pairs(50, 100, 20, 256, 1, 3, path=path, operator=True) is False
    assert autotune.lookup_pairs(50, 100, 20, 256, 1, 3, path=path) is True


def test_matrix_shape_default_and_missing_cache(tmp_path):
    path = _cache(tmp_path, {"N50-C3-K128-T2048-chi64-grad": {"warps": 6, "ctas_per_sm": 1}})
    assert autotune.lookup_pairs(50, 100, 64, 256, 8, 3, path=path) is True     # entry without "pairs"
    assert autotune.lookup_pairs(8, 20, 16, 16, 4, 2, path=path) is True        # nothing cached
    missing = str(tmp_path / "absent.json")
    assert autotune.lookup(50, 100, 64, 256, 8, 3, path=missing) == (0, 0)
    assert autotune.lookup_pairs(50, 100, 64, 256, 8, 3, path=missing) is True


def test_shipped_cache_covers_the_benchmark_and_the_gate_workload():
    cache = autotune.load()
    for key, args, op in (("N50-C3-K128-T2048-chi64-grad", (50, 100, 64, 256, 8, 3), False),
                          ("N50-C3-K128-T256-chi32-grad-op", (50, 100, 20, 256, 1, 3), True)):
        e = cache[key]
        assert autotune.lookup(*args, operator=op) == (e["warps"], e["ctas_per_sm"])
        # the cached choice is the fastest of the shapes it timed
        best = min(e["ms"], key=e["ms"].get)
        assert best == "%dx%d" % (e["warps"], e["ctas_per_sm"]) + ("" if e.get("pairs", True) else "-warp")
