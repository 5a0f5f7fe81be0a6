"""Autotuner for the batched training step.

Candidates are tuples of trainer settings: (blend variant, views per step)
and optionally the chunk length of the blend schedule (list entries per
chunk job: long lists favour longer chunks).  Each candidate builds its
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
    """make_trainer(*candidate) -> trainer with ``.step()`` and ``.units``; a candidate is
    (variant, views_per_step) or (variant, views_per_step, chunk).

    Returns (best candidate tuple, table of {candidate: units/s}).  The trainers are rebuilt from the
    same initial state by ``make_trainer``; state changes made while timing are the caller's to discard."""
    dev = torch.cuda.get_device_name()
    full = f"{dev}|{key}"
    cache = _load_cache() if use_cache else {}
    if full in cache:
        c = cache[full]
        return tuple(c["best"]), c["table"]
    table = {}
    for cand in (candidates or DEFAULT_CANDIDATES):
        tr = make_trainer(*cand)
        sec = time_trainer(tr, steps, warmup)
        table[",".join(str(x) for x in cand)] = tr.units.n / sec
        del tr
        torch.cuda.empty_cache()
    best = tuple(int(x) for x in max(table, key=table.get).split(","))
    cache[full] = {"best": list(best), "table": table}
    _save_cache(cache)
    return best, table
