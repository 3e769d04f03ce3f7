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
    assert A.choose({(32, 32, 1, 0.0): 3.0, (16, 16, 4, 0.0): 2.0, (64, 32, 1, 0.0): 2.0}) == (16, 16, 4, 0.0)
    assert A.choose({}) is None


def test_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setenv("RF_AUTOTUNE_CACHE", str(tmp_path / "at.json"))
    assert A.lookup("GB300", 2048, 2048) is None
    A.record("GB300", 2048, 2048, 32, 16, 1, 0.0, 27.5, {"32x16x1x0": 27.5})
    A.record("GB300", 500, 512, 16, 0, 8, 2.0, 3.0)
    assert A.lookup("GB300", 2000, 1500) == (32, 16, 1, 0.0)
    assert A.lookup("GB300", 300, 512) == (16, 0, 8, 2.0)
    assert A.lookup("other", 2048, 2048) is None
    d = json.load(open(tmp_path / "at.json"))
    assert d["GB300"]["2048"]["timings"] == {"32x16x1x0": 27.5}


def test_entries_without_window_read_as_default(tmp_path, monkeypatch):
    monkeypatch.setenv("RF_AUTOTUNE_CACHE", str(tmp_path / "at.json"))
    json.dump({"GB300": {"2048": {"band": 32, "block": 32, "variant": 2, "ms": 13.0}}}, open(tmp_path / "at.json", "w"))
    assert A.lookup("GB300", 2048, 2048) == (32, 32, 2, 0.0)


def test_entries_without_variant_are_ignored(tmp_path, monkeypatch):
    monkeypatch.setenv("RF_AUTOTUNE_CACHE", str(tmp_path / "at.json"))
    json.dump({"GB300": {"2048": {"band": 32, "block": 32, "ms": 27.5}}}, open(tmp_path / "at.json", "w"))
    assert A.lookup("GB300", 2048, 2048) is None


def test_candidates_are_accepted_shapes():
    # every candidate fits its kernel's shape rules: the tile queue takes
    # tile sides 16 and 32 and a non-negative window; for the line sweeps K a
    # power of two in [4, 32], R >= K, R + 2K <= 96 for one thread per node,
    # <= 128 for four; the streamed kernel is compiled for four (R, K) shapes
    for band, block, variant, window in A.CANDIDATES:
        assert variant in (1, 2, 4, 8) and window >= 0.0
        if variant == 8:
            assert band in (16, 32)
            continue
        assert window == 0.0
        assert block in (4, 8, 16, 32) and band >= block
        assert band + 2 * block <= (128 if variant == 4 else 96)
        if variant == 2:
            assert (band, block) in {(32, 32), (64, 16), (32, 16), (16, 16)}


def test_batch_candidates_and_key():
    # tile queue (variant 8) with tile side 16 or 32, or the persistent kernel (variant 1)
    for band, variant, window in A.BATCH_CANDIDATES:
        assert (variant == 8 and band in (16, 32) and window >= 0.0) or (variant == 1 and window == 0.0)
    assert A.batch_key(256, 62834981) == "batch256x67108864"
