"""Autotuner for the screen-tile shape and the K-buffer layout of a render configuration.

Results depend on neither (a Gaussian takes part at a pixel by a per-pixel test, not by
tile membership; the walk keeps the same Top-K whether its K-buffer lives in registers
or in shared memory), so both are pure performance choices.  For a given configuration
-- cameras, Gaussian count, K, D, feature dtype -- every compiled (shape, layout) pair is
timed on the full training step replayed as a CUDA graph, and the fastest is cached in a
JSON file keyed by the configuration.  K itself is a model parameter (it changes the
rendered feature), so it is part of the key, never tuned.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Dict, Sequence

import torch

TILE_SHAPES = [(16, 16), (32, 8), (16, 8), (8, 8)]
# where the walk keeps each pixel's Top-K (gs_config.topk_layout): registers, shared memory
KBUF_LAYOUTS = {"reg": 0, "smem": 1, "warp": 2}
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


def layouts_for(K: int) -> Dict[str, int]:
    """The K-buffer layouts compiled for K (the shared-memory forms hold K <= 16)."""
    return {n: v for n, v in KBUF_LAYOUTS.items() if v == 0 or K <= 16}


def tune(cameras, n_gauss: int, K: int, D: int, feat_dtype: str, step_factory, cache_path: str = DEFAULT_CACHE,
         shapes=TILE_SHAPES, layouts=None, force: bool = False) -> Dict:
    """step_factory(tile, layout) -> callable running one training step with that tile
    shape and K-buffer layout.  Returns {"tile": (w, h), "layout": name, "ms": {"WxH/name":
    ms}} and caches it."""
    key = config_key(cameras, n_gauss, K, D, feat_dtype)
    cache = load_cache(cache_path)
    if not force and key in cache and "layout" in cache[key]:
        hit = cache[key]
        return {"tile": tuple(hit["tile"]), "layout": hit["layout"], "ms": hit["ms"], "cached": True}
    layouts = layouts_for(K) if layouts is None else layouts
    ms = {}
    for shape in shapes:
        for name, value in layouts.items():
            ms[f"{shape[0]}x{shape[1]}/{name}"] = time_step(lambda: step_factory(shape, value))
            torch.cuda.empty_cache()
    best = min(ms, key=ms.get)
    shape_s, layout = best.split("/")
    tile = tuple(int(v) for v in shape_s.split("x"))
    cache[key] = {"tile": list(tile), "layout": layout, "ms": ms}
    save_cache(cache, cache_path)
    return {"tile": tile, "layout": layout, "ms": ms, "cached": False}
