"""Autotuner for the batched training step.

Candidates are (blend variant, views per step).  Each candidate builds its
trainer, captures its CUDA graph, and is timed over a few replays with CUDA
events; throughput is (partition, view) units per second.  The winner is
cached per GPU and workload in ``_build/tune_cache.json``.
"""
from __future__ import annotations

import json
import os

import torch

from . import build as _build

CACHE = os.path.join(_build.BUILD, "tune_cache.json")
DEFAULT_CANDIDATES = [(v, k) for k in (1, 2) for v in (0, 1, 2)]


def _load_cache():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _save_cache(c):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def time_trainer(tr, steps: int = 6, warmup: int = 2) -> float:
    """Seconds per step of a trainer (graph replays when it uses a graph)."""
    for _ in range(warmup):
        tr.step()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        tr.step()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps / 1e3


def autotune(make_trainer, key: str, candidates=None, steps: int = 6, warmup: int = 2, use_cache: bool = True):
    """make_trainer(variant, views_per_step) -> trainer with ``.step()`` and ``.units``.

    Returns (best (variant, views_per_step), table of {candidate: units/s}).  The trainers are
    rebuilt from the same initial state by ``make_trainer``; state changes made while timing are
    the caller's to discard."""
    dev = torch.cuda.get_device_name()
    full = f"{dev}|{key}"
    cache = _load_cache() if use_cache else {}
    if full in cache:
        c = cache[full]
        return (c["variant"], c["views_per_step"]), c["table"]
    table = {}
    for (variant, vps) in (candidates or DEFAULT_CANDIDATES):
        tr = make_trainer(variant, vps)
        sec = time_trainer(tr, steps, warmup)
        table[f"{variant},{vps}"] = tr.units.n / sec
        del tr
        torch.cuda.empty_cache()
    best = max(table, key=table.get)
    variant, vps = (int(x) for x in best.split(","))
    cache[full] = {"variant": variant, "views_per_step": vps, "table": table}
    _save_cache(cache)
    return (variant, vps), table
