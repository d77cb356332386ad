"""Voxel-tile autotuner: candidate shapes and cache (CPU), tuning runs (GPU)."""
import json
import os

import pytest

import synth
from synth import MM
from paper_2512_11086_gb300 import tune


def test_candidates_for_a_bscan_keep_one_row_layer():
    g = synth.full_bscan_geometry()
    c = tune.candidate_tiles(g)
    assert (64, 1, 16) in c and (128, 1, 8) in c and (32, 1, 32) in c
    assert all(t[1] == 1 and t[0] * t[1] * t[2] == 1024 for t in c)


def test_candidates_for_a_volume_split_rows():
    g = synth.hercules_volume_geometry()
    c = tune.candidate_tiles(g)
    assert (32, 4, 8) in c and (64, 2, 8) in c and (128, 8, 1) in c
    assert all(t[0] * t[1] * t[2] == 1024 for t in c)


def test_geometry_key_separates_classes():
    a = tune.geometry_key(synth.full_bscan_geometry(), "f16")
    b = tune.geometry_key(synth.full_bscan_geometry(), "f32")
    c = tune.geometry_key(synth.tiny_bscan_geometry(), "f16")
    assert len({a, b, c}) == 3
    assert a == tune.geometry_key(synth.full_bscan_geometry(), "f16")


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "sub" / "tiles.json")
    tune._store(p, {"k": {"best": [64, 1, 16]}})
    assert tune._load(p) == {"k": {"best": [64, 1, 16]}}
    assert tune._load(str(tmp_path / "missing.json")) == {}


@pytest.mark.gpu
def test_tune_tile_and_stream_on_gpu(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11086_gb300 import build
    build.build()
    cache = str(tmp_path / "tiles.json")
    g = synth.Geometry(n_tx=32, n_ch=32, n_samples=1024, out_dims=(256, 1, 512),
                       out_min=(-3 * MM, 0.0, 4 * MM), out_max=(3 * MM, 0.0, 16 * MM))
    best = tune.tune_tile(g, "f16", cache_path=cache, reps=2)
    assert best in tune.candidate_tiles(g)
    data = json.load(open(cache))
    assert list(best) == data[tune.geometry_key(g, "f16")]["best"]
    assert tune.tune_tile(g, "f16", cache_path=cache) == best          # served from the cache
    g2 = synth.Geometry(n_tx=64, n_ch=32, n_samples=2048, out_dims=(128, 1, 256),
                        out_min=(-3 * MM, 0.0, 4 * MM), out_max=(3 * MM, 0.0, 16 * MM))
    tiles = tune.tune_stream([g, g2, g], "f16", cache_path=cache, reps=2)
    assert len(tiles) == 3 and tiles[0] == tiles[2] == best
    assert tiles[1] in tune.candidate_tiles(g2)
