"""Autotuner for the screen-tile shape of a render configuration.

Results do not depend on the tile shape (a Gaussian takes part at a pixel by a per-pixel
test, not by tile membership), so the tile shape is a pure performance choice.  For a
given configuration -- cameras, Gaussian count, K, D, feature dtype -- every compiled
shape is timed on the full training step replayed as a CUDA graph, and the fastest is
cached in a JSON file keyed by the configuration.  K itself is a model parameter (it
changes the rendered feature), so it is part of the key, never tuned.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Dict, Sequence

import torch

TILE_SHAPES = [(16, 16), (32, 8), (16, 8), (8, 8)]
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json")


def config_key(cameras: Sequence, n_gauss: int, K: int, D: int, feat_dtype: str) -> str:
    cams = ";".join(f"{int(c.width)}x{int(c.height)}" for c in cameras)
    raw = f"{torch.cuda.get_device_name()}|{cams}|N={n_gauss}|K={K}|D={D}|{feat_dtype}"
    return hashlib.sha1(raw.encode()).hexdigest()[:16] + "|" + raw


def load_cache(path: str = DEFAULT_CACHE) -> Dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save_cache(cache: Dict, path: str = DEFAULT_CACHE):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_step(make_step, reps: int = 10, warmup: int = 3) -> float:
    """Milliseconds per replay of the graph-captured step built by make_step()."""
    step = make_step()
    stream = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        step()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(cameras, n_gauss: int, K: int, D: int, feat_dtype: str, step_factory, cache_path: str = DEFAULT_CACHE,
         shapes=TILE_SHAPES, force: bool = False) -> Dict:
    """step_factory(tile) -> callable running one training step with that tile shape.
    Returns {"tile": (w, h), "ms": {shape: ms}} and caches it."""
    key = config_key(cameras, n_gauss, K, D, feat_dtype)
    cache = load_cache(cache_path)
    if not force and key in cache:
        hit = cache[key]
        return {"tile": tuple(hit["tile"]), "ms": hit["ms"], "cached": True}
    ms = {}
    for shape in shapes:
        ms[f"{shape[0]}x{shape[1]}"] = time_step(lambda: step_factory(shape))
        torch.cuda.empty_cache()
    best = min(ms, key=ms.get)
    tile = tuple(int(v) for v in best.split("x"))
    cache[key] = {"tile": list(tile), "ms": ms}
    save_cache(cache, cache_path)
    return {"tile": tile, "ms": ms, "cached": False}
