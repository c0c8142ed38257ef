"""Host logic of the autotuner (no GPU): class keys, candidate constraints, cache."""
import json

from paper_1011_2807_gb300 import autotune


def test_class_key_buckets():
    a = autotune.class_key(1_000_000, 5000, 150.0, 5, "u8")
    b = autotune.class_key(1_100_000, 5200, 160.0, 5, "u8")
    c = autotune.class_key(100_000, 5000, 150.0, 5, "u8")
    assert a == b and a != c and a.startswith("u8:")


def test_candidates_respect_the_kernel_limits():
    for n_s in (5000, 200000, 3_000_000):
        cs = autotune.candidates(n_s)
        assert cs
        for c in cs:
            assert 4 * c["threads"] <= c["block_size"] <= 64 * c["threads"]
            assert c["block_size"] <= 2 * max(2048, n_s)
    assert all(c["threads"] == 512 for c in autotune.candidates(10**6, threads=512))


def test_heuristic_and_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setenv("KNN_TUNE_CACHE", str(tmp_path / "tune.json"))
    assert autotune.heuristic(3000)["block_size"] == 4096
    assert autotune.heuristic(10**7)["block_size"] == 16384
    key = autotune.class_key(50000, 300, 120, 10, "u8")
    autotune._store({key: {"block_size": 8192, "threads": 256, "blocks_per_launch": 4}})
    got = autotune.lookup(50000, 300, 120, 10, "u8")
    assert got["block_size"] == 8192 and got["threads"] == 256
    assert got["level_margin"] == autotune.DEFAULT["level_margin"]   # entries cached without a margin
    assert json.load(open(tmp_path / "tune.json"))[key]["blocks_per_launch"] == 4
    # an unseen class falls back to the heuristic
    assert autotune.lookup(12, 1, 1, 1, "f32")["block_size"] == 2048
