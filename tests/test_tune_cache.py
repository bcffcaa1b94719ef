"""The autotuner's cache: keys, persistence, and the hit / miss paths (with a fake tuner; no GPU)."""
import json

import pytest

from paper_1905_07224_gb300 import tune_cache as tc


def test_keys_bucket_by_gpu_level_and_size():
    assert tc.cache_key("GB300", 4, 134_000_000) == "GB300|xfl4|2^26"
    assert tc.cache_key("GB300", 4, 134_000_000) == tc.cache_key("GB300", 4, 100_000_000)
    assert tc.cache_key("GB300", 2, 134_000_000) != tc.cache_key("GB300", 4, 134_000_000)
    assert tc.cache_key("GB300", 0, 1 << 31) == "GB300|xfl0|2^31"
    assert tc.cache_key("X", 0, 0) == "X|xfl0|2^0"


class FakePgz:
    """Stands in for the binding: records calls, returns a fixed choice."""
    def __init__(self):
        self.tuned, self.applied = 0, []

    def pgz_autotune(self, ctx, jobs, chunks, wpbs, reps, sweep_exec=False):
        self.tuned += 1
        return 0, [], {"chunk_bytes": 131072, "warps_per_block": 8, "exec_pipelined": 1, "status": 0, "ms": 10.8}

    def pgz_set_tuning(self, ctx, chunk_bytes, wpb, pipe):
        self.applied.append((chunk_bytes, wpb, pipe))
        return 0


def test_miss_tunes_and_stores_then_hit_applies(tmp_path):
    path = str(tmp_path / "tune.json")
    fake = FakePgz()
    key = tc.cache_key("GB300", 4, 268_000_000)
    st, e, hit = tc.autotune_cached(fake, 1, [], key, tc.TuneCache(path), [65536, 131072], [2, 4, 8])
    assert st == 0 and not hit and fake.tuned == 1 and fake.applied == []
    assert json.load(open(path))[key] == {"chunk_bytes": 131072, "warps_per_block": 8, "exec_pipelined": 1,
                                          "ms": 10.8}
    # a new process: the file is read back and the choice applied without timing
    st, e, hit = tc.autotune_cached(fake, 2, [], key, tc.TuneCache(path), [65536], [4])
    assert st == 0 and hit and fake.tuned == 1 and fake.applied == [(131072, 8, 1)]
    # another level misses
    st, e, hit = tc.autotune_cached(fake, 2, [], tc.cache_key("GB300", 2, 268_000_000), tc.TuneCache(path),
                                    [65536], [4])
    assert not hit and fake.tuned == 2 and len(json.load(open(path))) == 2


def test_a_failed_tuning_is_not_stored(tmp_path):
    class Failing(FakePgz):
        def pgz_autotune(self, *a, **k):
            return 3, [], None
    path = str(tmp_path / "tune.json")
    st, e, hit = tc.autotune_cached(Failing(), 1, [], "k", tc.TuneCache(path), [65536], [4])
    assert st == 3 and e is None and not hit
    assert not (tmp_path / "tune.json").exists()


def test_a_foreign_file_is_rejected(tmp_path):
    p = tmp_path / "tune.json"
    p.write_text("[1, 2]")
    with pytest.raises(ValueError):
        tc.TuneCache(str(p))
