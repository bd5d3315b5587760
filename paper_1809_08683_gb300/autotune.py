"""Launch-shape autotuner for the fused collide-stream kernel.

The fused kernel gives each CTA a strip of ``bx`` columns (32, 64 or 128
threads) and a run of ``by`` rows that it sweeps with a three-row ring of
rho' and p' in shared memory.  Short runs give more CTAs (better SM fill on
small lattices) but re-read two halo rows per run; long runs amortise the
halo but may leave SMs idle.  The best shape depends on the lattice shape and
the precision, so it is measured: every candidate is timed with CUDA events
on the lattice's own stream, and the winner is cached per
(precision, nx class, ny class) in a JSON file.
"""
from __future__ import annotations

import json
import os
import threading

from . import lbm

_CACHE_PATH = os.environ.get(
    "LBM_TUNE_CACHE", os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tile_cache.json"))
_lock = threading.Lock()
BX_CANDIDATES = (32, 64, 128)
BY_CANDIDATES = (4, 8, 16, 32, 64, 128)


def size_class(n: int) -> int:
    """Round a lattice extent up to the next power of two (>= 16)."""
    c = 16
    while c < n:
        c *= 2
    return c


def key_for(cfg: dict) -> str:
    return f"p{int(cfg.get('precision', 0))}_x{size_class(cfg['nx'])}_y{size_class(cfg['ny'])}"


def _load():
    try:
        with open(_CACHE_PATH) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _store(d):
    os.makedirs(os.path.dirname(_CACHE_PATH), exist_ok=True)
    tmp = _CACHE_PATH + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, _CACHE_PATH)


PAIR_BX_CANDIDATES = (64, 128, 256)
WARP_BX_CANDIDATES = (30, 60, 120)
WARP2_BX_CANDIDATES = (60, 120, 240)


def candidates(cfg: dict):
    """(bx, by, pair) shapes worth timing for this lattice: one node per
    thread in block strips or warp strips for every precision, two nodes per
    thread for FP32 storage."""
    shapes = [(bx, 0) for bx in BX_CANDIDATES] + [(bx, 4) for bx in WARP_BX_CANDIDATES]
    if int(cfg.get("precision", 0)) == 1:
        shapes += [(bx, 3) for bx in BX_CANDIDATES]
        shapes += [(bx, pr) for bx in PAIR_BX_CANDIDATES for pr in (1, 2)]
        shapes += [(bx, 5) for bx in WARP2_BX_CANDIDATES]
    out = []
    for bx, pr in shapes:
        if bx > 32 and cfg["nx"] <= bx // 2:
            continue
        for by in BY_CANDIDATES:
            if by > cfg["ny"] and by != BY_CANDIDATES[0]:
                continue
            out.append((bx, by, pr))
    return out


def measure(cfg: dict, bx: int, by: int, pair: int = 0, steps: int = 20, stream=None) -> float:
    """MLUPS of the fused kernel alone for one launch shape."""
    lat = lbm.Lattice(cfg, stream=stream)
    lat.set_tile(bx, by, pair)
    batch = lbm.Batch([lat], graph_steps=0)
    batch.step_profiled(4)                       # warm-up
    ms, _ = batch.step_profiled(steps)
    batch.close()
    lat.close()
    return cfg["nx"] * cfg["ny"] * steps / (ms * 1e-3) / 1e6


def tune(cfg: dict, steps: int = 20, force: bool = False, stream=None) -> tuple:
    """Best (bx, by, pair) for this configuration's class, measured on first use."""
    key = key_for(cfg)
    with _lock:
        cache = _load()
        if key in cache and not force and len(cache[key]["tile"]) == 3:
            return tuple(cache[key]["tile"])
    results = {}
    for bx, by, pr in candidates(cfg):
        results[(bx, by, pr)] = measure(cfg, bx, by, pr, steps, stream)
    best = max(results, key=results.get)
    with _lock:
        cache = _load()
        cache[key] = {"tile": list(best), "mlups": results[best],
                      "all": {f"{b[0]}x{b[1]}p{b[2]}": v for b, v in results.items()}}
        _store(cache)
    return best


def apply(lattices, steps: int = 20):
    """Set every lattice's launch shape from the cache, tuning unseen classes."""
    for lat in lattices:
        bx, by, pr = tune(lat.cfg, steps=steps, stream=lat.stream)
        lat.set_tile(bx, by, pr)


# Shapes tried for a whole batch: paired block strips with run lengths
# around the built-in batch length, block strips, and the built-in default
# (None: each member's default shape, runs shortened by the batch builder).
BATCH_SHAPES = (None, (128, 16, 1), (128, 24, 1), (128, 32, 1), (128, 48, 1), (256, 32, 1), (128, 24, 0))


def measure_batch(lattices, shape, steps: int = 10, warmup: int = 3) -> float:
    """Milliseconds per time step of the whole batch (fused and wall-pass
    launches, CUDA events) with `shape` applied to every member, or each
    member's default shape for None.  The shape stays applied."""
    for lat in lattices:
        if shape is None:
            lat.set_tile(0, 0, 0)
        else:
            lat.set_tile(*shape)
    batch = lbm.Batch(lattices, graph_steps=0)
    batch.step_profiled(warmup)
    a, b = batch.step_profiled(steps)
    batch.close()
    return (a + b) / steps


def tune_batch(lattices, shapes=BATCH_SHAPES, steps: int = 10):
    """Time the batch under every candidate shape that all members accept
    and leave the fastest applied.  Returns (best, {shape: ms per step});
    None stands for the built-in default."""
    results = {}
    for shape in shapes:
        if shape is not None:
            if shape[2] in (1, 2, 3, 5) and any(int(l.cfg.get("precision", 0)) != 1 for l in lattices):
                continue
        results[shape] = measure_batch(lattices, shape, steps)
    best = min(results, key=results.get)
    for lat in lattices:
        if best is None:
            lat.set_tile(0, 0, 0)
        else:
            lat.set_tile(*best)
    return best, results
