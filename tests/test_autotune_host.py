"""Autotuner host logic without a GPU: shape buckets and the JSON cache."""
import json

from paper_2605_27147_gb300 import autotune


def test_shape_key_buckets_half_octaves():
    k = autotune.shape_key("GB300", 4096, 522117394, 1047006)
    assert k.startswith(f"v{autotune.CACHE_VERSION}|GB300|")
    # within half an octave the key is the same, across it it differs
    assert autotune.shape_key("GB300", 4096, 522117394, 1047006) == autotune.shape_key("GB300", 4100, 5.22e8, 1.05e6)
    assert autotune.shape_key("GB300", 4096, 5.22e8, 1.05e6) != autotune.shape_key("GB300", 8192, 5.22e8, 1.05e6)
    assert autotune.shape_key("GB300", 1, 0, 0) == f"v{autotune.CACHE_VERSION}|GB300|c0|t0|m0"
    assert autotune.shape_key("A", 8, 8, 8) != autotune.shape_key("B", 8, 8, 8)   # per GPU model


def test_cache_file_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "autotune.json"
    monkeypatch.setenv("PS_AUTOTUNE_CACHE", str(path))
    assert autotune._load_file() == {}                 # no file yet
    entry = {"tile_log2": 12, "ms": 38.6, "trials": [], "shape": "k"}
    autotune._store_file({"k": entry})
    assert json.loads(path.read_text()) == {"k": entry}
    assert autotune._load_file() == {"k": entry}
    path.write_text("{not json")                       # a damaged cache reads as empty
    assert autotune._load_file() == {}


def test_candidates_cover_every_tile_size():
    assert set(autotune.TILE_LOG2) == {10, 11, 12}
    assert set(autotune.MERGE_LANES) == {4, 8, 16}
