"""Voxel-tile autotuner for the tiled DAS.

A tile is (bu, bv, bw) with bu*bv*bw = 1024 voxels: bu (32, 64 or 128) runs
along the image axis parallel to the transmit line elements, bv along the
other lateral axis, bw along z. The plan's default comes from a geometric
model (shortest window in the largest window class); the autotuner instead
times every admissible shape with the library's own DAS on the GPU (CUDA
events, after warm-up) and keeps the fastest. Results are cached in a JSON
file keyed by the geometry, so a frame class is tuned once.

A batch runs the frames of each window class and tile extent as their own
persistent launch, so ``tune_stream`` gives every distinct frame class its own
fastest tile.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

from . import Plan, make_params, DAS_TILED

Tile = Tuple[int, int, int]
_lock = threading.Lock()


def default_cache_path() -> str:
    base = os.environ.get("RCBF_TUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "rcbf", "tiles.json")


def geometry_key(g, decoded_dtype: str) -> str:
    fields = (int(g.n_tx), int(g.n_ch), int(g.n_samples), tuple(int(v) for v in g.out_dims),
              tuple(round(float(v), 9) for v in g.out_min), tuple(round(float(v), 9) for v in g.out_max),
              int(g.tx_orientation), int(g.rx_orientation), round(float(g.fs), 3), round(float(g.c), 6),
              round(float(g.t0), 12), round(float(g.tx_pitch), 9), round(float(g.rx_pitch), 9),
              round(float(g.f_number), 6), decoded_dtype, str(getattr(g, "interp", "linear")))
    return repr(fields)


def candidate_tiles(g, bus: Iterable[int] = (32, 64, 128)) -> List[Tile]:
    out = []
    # the lane axis is x for row transmit elements, y for column ones
    lane_is_x = int(g.tx_orientation) == 0
    other = int(g.out_dims[1]) if lane_is_x else int(g.out_dims[0])
    for bu in bus:
        rows = 1024 // bu
        bv = 1
        while bv <= rows:
            if bv == 1 or other > 1:
                out.append((bu, bv, rows // bv))
            bv *= 2
    return out


def _load(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, data: Dict[str, dict]) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_tiles(g, decoded_dtype: str = "f16", tiles: Optional[Sequence[Tile]] = None, reps: int = 5,
               warmup: int = 2) -> Dict[Tile, float]:
    """Milliseconds per DAS call for each admissible tile (tiled form only)."""
    import torch
    tiles = list(tiles) if tiles is not None else candidate_tiles(g)
    tdt = {"f16": torch.float16, "f32": torch.float32, "cf32": torch.float32}[decoded_dtype]
    planes = (2,) if decoded_dtype == "cf32" else ()       # complex data: two real planes
    dec = torch.randn(planes + (int(g.n_tx), int(g.n_ch), int(g.n_samples)), device="cuda").to(tdt)
    out = torch.empty(planes + (int(g.out_dims[2]), int(g.out_dims[1]), int(g.out_dims[0])), device="cuda")
    result: Dict[Tile, float] = {}
    for t in tiles:
        plan = Plan(make_params(g, decoded_dtype=decoded_dtype, das_variant=DAS_TILED, tile=t))
        info = plan.info()
        if not info["tiled"]:
            continue
        for _ in range(warmup):
            plan.das(dec, out=out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            plan.das(dec, out=out)
        e1.record()
        torch.cuda.synchronize()
        result[tuple(t)] = e0.elapsed_time(e1) / reps
        plan.close()
    return result


def tune_tile(g, decoded_dtype: str = "f16", cache_path: Optional[str] = None, reps: int = 5) -> Tile:
    """Fastest tile for one geometry (cached)."""
    path = cache_path or default_cache_path()
    key = geometry_key(g, decoded_dtype)
    with _lock:
        cache = _load(path)
        if key in cache:
            return tuple(cache[key]["best"])
    times = time_tiles(g, decoded_dtype, reps=reps)
    if not times:
        raise RuntimeError("no tile admits the tiled DAS for this geometry")
    best = min(times, key=times.get)
    with _lock:
        cache = _load(path)
        cache[key] = {"best": list(best), "ms": {"%d,%d,%d" % t: v for t, v in times.items()}}
        _store(path, cache)
    return best


def tune_stream(geometries: Sequence, decoded_dtype: str = "f16", cache_path: Optional[str] = None,
                reps: int = 3) -> List[Tile]:
    """Tiles for the frames of a batch: the fastest tile of each frame class
    (a batch runs the frames of each window class and tile extent along u as
    their own persistent launch, so the classes need not share a tile)."""
    path = cache_path or default_cache_path()
    classes: Dict[str, Tuple[object, int]] = {}
    for g in geometries:
        k = geometry_key(g, decoded_dtype)
        classes[k] = (g, classes[k][1] + 1 if k in classes else 1)
    per_class: Dict[str, Dict[Tile, float]] = {}
    for k, (g, _) in classes.items():
        with _lock:
            cache = _load(path)
        if k in cache and "ms" in cache[k]:
            per_class[k] = {tuple(int(v) for v in t.split(",")): ms for t, ms in cache[k]["ms"].items()}
        else:
            per_class[k] = time_tiles(g, decoded_dtype, reps=reps)
            with _lock:
                cache = _load(path)
                best = min(per_class[k], key=per_class[k].get)
                cache[k] = {"best": list(best), "ms": {"%d,%d,%d" % t: v for t, v in per_class[k].items()}}
                _store(path, cache)
    tiles = []
    for g in geometries:
        opts = per_class[geometry_key(g, decoded_dtype)]
        if not opts:
            raise RuntimeError("no tile admits the tiled DAS for a frame of the batch")
        tiles.append(min(opts, key=opts.get))
    return tiles
