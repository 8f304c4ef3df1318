"""Autotuner cache: stored per (GPU, workload) key, applied on a hit, re-tuned
on a miss or an unusable entry (no GPU: the library calls are faked)."""

import json
import os

import pytest

from paper_2305_07083_gb300 import dfb as D
from paper_2305_07083_gb300 import tuning


class FakeLib:
    def __init__(self, fail_set=False):
        self.tuned = 0
        self.applied = []
        self.fail_set = fail_set

    def dfb_graph_autotune(self, g, stream, reps):
        self.tuned += 1
        return {"ring_kb": 72, "ctas_per_sm": 3, "groups": 1, "ms": 2.5}

    def dfb_graph_set_tuning(self, g, ring, ctas, groups):
        if self.fail_set:
            raise D.DfbError(D.DFB_ERR_INVALID_ARG, "dfb_graph_set_tuning")
        self.applied.append((ring, ctas, groups))


def test_miss_then_hit(tmp_path):
    path = str(tmp_path / "t.json")
    key = tuning.make_key("GB300/sm_103/152", {"frames": [[2048, 2048]], "T": 64, "dtype": "f16"})
    lib = FakeLib()
    first = tuning.autotune_cached("g", key, path=path, lib=lib)
    assert first["cached"] is False and lib.tuned == 1
    second = tuning.autotune_cached("g", key, path=path, lib=lib)
    assert second["cached"] is True and lib.tuned == 1
    assert lib.applied == [(72, 3, 1)]
    other = tuning.make_key("GB300/sm_103/152", {"frames": [[1024, 1024]], "T": 64, "dtype": "f16"})
    tuning.autotune_cached("g", other, path=path, lib=lib)
    assert lib.tuned == 2
    assert len(json.load(open(path))) == 2


def test_unusable_entry_is_retuned(tmp_path):
    path = str(tmp_path / "t.json")
    key = tuning.make_key("gpu", {"w": 1})
    tuning.store(key, {"ring_kb": 300, "ctas_per_sm": 9, "groups": 9, "ms": 1.0}, path)
    lib = FakeLib(fail_set=True)
    got = tuning.autotune_cached("g", key, path=path, lib=lib)
    assert got["cached"] is False and lib.tuned == 1
    assert json.load(open(path))[key]["ring_kb"] == 72


def test_corrupt_file_is_ignored(tmp_path):
    path = tmp_path / "t.json"
    path.write_text("{not json")
    assert tuning.load(str(path)) == {}
    key = tuning.make_key("gpu", {"w": 2})
    got = tuning.autotune_cached("g", key, path=str(path), lib=FakeLib())
    assert got["cached"] is False
    assert key in json.load(open(path))


def test_failed_store_leaves_the_file_and_no_temporary(tmp_path):
    path = str(tmp_path / "t.json")
    tuning.store("a", {"ring_kb": 110, "ctas_per_sm": 2, "groups": 2, "ms": 1.0}, path)
    before = open(path).read()
    with pytest.raises(TypeError):
        tuning.store("b", {"ring_kb": object(), "ctas_per_sm": 2, "groups": 2}, path)   # not JSON
    assert open(path).read() == before
    assert sorted(os.listdir(tmp_path)) == ["t.json"]
