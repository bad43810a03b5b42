"""The autotuner's shape file (paper_1108_1954_gb300.tune_cache) on the CPU:
power-of-two buckets, keys that separate runs of another kind, and a file
that round-trips, survives a bad entry and is replaced whole."""
import json
import os

from paper_1108_1954_gb300 import tune_cache as tc


def test_buckets():
    assert [tc.bucket(n) for n in (1, 2, 3, 4, 5, 64, 65, 4096, 1 << 26)] == \
        [1, 2, 4, 4, 8, 64, 128, 4096, 1 << 26]


def test_keys_separate_runs_of_another_kind():
    k = tc.key("NVIDIA GB300", 1 << 26, 4096, 20, 0, 0)
    assert k == tc.key("NVIDIA GB300 ", (1 << 25) + 1, 4000, 20, 0, 0)     # same buckets
    others = [tc.key("NVIDIA B200", 1 << 26, 4096, 20, 0, 0),
              tc.key("NVIDIA GB300", 1 << 27, 4096, 20, 0, 0),
              tc.key("NVIDIA GB300", 1 << 26, 8192, 20, 0, 0),
              tc.key("NVIDIA GB300", 1 << 26, 4096, 0, 0, 0),
              tc.key("NVIDIA GB300", 1 << 26, 4096, 20, 2, 0),
              tc.key("NVIDIA GB300", 1 << 26, 4096, 20, 0, 1)]
    assert len(set(others + [k])) == 7


def test_store_lookup_and_replace(tmp_path):
    path = str(tmp_path / "shapes.json")
    assert tc.lookup(path, "a") is None                        # no file yet
    tc.store(path, "a", 8, 512, 1, 0.1777)
    tc.store(path, "b", 9, 512, 2, 0.1783)
    assert tc.lookup(path, "a") == {"variant": 8, "block": 512, "unroll": 1, "ms": 0.1777}
    tc.store(path, "a", 9, 768, 1, 0.17)                       # replaced, b kept
    assert tc.lookup(path, "a")["block"] == 768 and tc.lookup(path, "b")["unroll"] == 2
    assert sorted(json.load(open(path))) == ["a", "b"]
    assert not [f for f in os.listdir(tmp_path) if f.startswith(".tune_cache.")]


def test_bad_files_and_entries(tmp_path):
    path = str(tmp_path / "shapes.json")
    open(path, "w").write("{not json")
    assert tc.load(path) == {} and tc.lookup(path, "a") is None
    open(path, "w").write(json.dumps({"a": {"variant": 8}}))   # incomplete entry
    assert tc.lookup(path, "a") is None
    tc.store(path, "c", 8, 512, 1, 0.2)                        # a bad file is rewritten
    assert tc.lookup(path, "c")["variant"] == 8
