"""Host logic of the line-tile autotuner: size buckets, choice of the
fastest shape, and the on-disk cache (no GPU needed)."""
import json

from paper_2603_00035_gb300 import autotune as A


def test_bucket_is_next_power_of_two():
    assert A.bucket(64, 64) == 64
    assert A.bucket(65, 10) == 128
    assert A.bucket(1000, 2048) == 2048
    assert A.bucket(1, 1) == 1


def test_choose_fastest_first_on_ties():
    assert A.choose({(32, 32): 3.0, (16, 16): 2.0, (64, 32): 2.0}) == (16, 16)
    assert A.choose({}) is None


def test_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setenv("RF_AUTOTUNE_CACHE", str(tmp_path / "at.json"))
    assert A.lookup("GB300", 2048, 2048) is None
    A.record("GB300", 2048, 2048, 32, 16, 27.5, {"32x16": 27.5})
    A.record("GB300", 500, 512, 16, 16, 3.0)
    assert A.lookup("GB300", 2000, 1500) == (32, 16)
    assert A.lookup("GB300", 300, 512) == (16, 16)
    assert A.lookup("other", 2048, 2048) is None
    d = json.load(open(tmp_path / "at.json"))
    assert d["GB300"]["2048"]["timings"] == {"32x16": 27.5}
