"""Host logic of the multi-GPU form: one process per GPU, partitions as independent units.

The partitions of the method (Sec. II, "Data Partitioning" / "Parallel Training") are independent
problems: each trains on its own Gaussians, views and masks with no communication.  Across GPUs they
are sharded with no collective on the data path; the only collectives are the timing reduction of a
measurement (max over ranks) and the merge (Sec. II, "Global Reconstruction"), which gathers every
rank's owned splats to the rank that renders them.

Nothing here launches GPU work; the collectives run on whatever backend the caller's process group
uses (NCCL on GPUs, gloo on the CPU in the tests).
"""
from __future__ import annotations

import time
from datetime import timedelta

import numpy as np
import torch


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s independent scene (weak scaling: every rank its own problem)."""
    return int(base_seed) + 1_000_003 * int(rank)


def assign_units(sizes, world: int) -> list[list[int]]:
    """Deterministic longest-processing-time assignment of units (e.g. partitions, weighted by their
    Gaussian counts) to `world` ranks: units in decreasing size, each to the least-loaded rank (ties to
    the lower rank).  Every rank computes the same assignment from the same sizes without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    sizes = np.asarray(sizes, dtype=np.int64)
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += int(sizes[i])
    for r in range(world):
        out[r].sort()
    return out


def partition_subset(offsets, parts) -> tuple[np.ndarray, np.ndarray]:
    """The Gaussians of partitions `parts` of a partition-major layout (partition k holds
    [offsets[k], offsets[k + 1])): their indices in partition order and the offsets of the sub-layout
    (the rank's own partition-major parameter planes)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    parts = [int(k) for k in parts]
    if any(k < 0 or k >= len(offsets) - 1 for k in parts) or len(set(parts)) != len(parts):
        raise ValueError(f"partitions {parts} not a subset of 0..{len(offsets) - 2}")
    idx = [np.arange(offsets[k], offsets[k + 1], dtype=np.int64) for k in parts]
    sizes = [len(a) for a in idx]
    sub = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return (np.concatenate(idx) if idx else np.zeros(0, np.int64)), sub


def reduce_max(values, device=None) -> list[float]:
    """Element-wise max over ranks of a few host scalars (the timing of a measurement); identity when
    torch.distributed is not initialised."""
    import torch.distributed as dist
    vals = [float(v) for v in values]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return vals
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_throughput(units_per_rank, t_max_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed divided by the slowest rank's time."""
    return float(sum(units_per_rank)) / (float(t_max_ms) * 1e-3)


def gather_owned(params: torch.Tensor, keep: torch.Tensor, dst: int = 0):
    """Merge exchange: every rank contributes the columns of its parameter planes `params` [planes, n, 4]
    whose `keep` flag is set (its owned Gaussians); rank `dst` receives all of them concatenated in rank
    order ([planes, total, 4]), the other ranks None.  Sizes travel first (all_gather), then the padded
    blocks (gather), so ranks may own different numbers of Gaussians."""
    import torch.distributed as dist
    mine = params[:, keep.to(torch.bool)].contiguous()
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return mine
    world, rank = dist.get_world_size(), dist.get_rank()
    n = torch.tensor([mine.shape[1]], dtype=torch.int64, device=params.device)
    counts = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts, n)
    counts = [int(c.item()) for c in counts]
    cap = max(max(counts), 1)
    pad = torch.zeros((params.shape[0], cap, params.shape[2]), dtype=params.dtype, device=params.device)
    pad[:, : mine.shape[1]] = mine
    if rank == dst:
        bufs = [torch.empty_like(pad) for _ in range(world)]
        dist.gather(pad, gather_list=bufs, dst=dst)
        return torch.cat([b[:, :c] for b, c in zip(bufs, counts)], dim=1)
    dist.gather(pad, dst=dst)
    return None


def init_group(backend: str, timeout_s: float = 300.0, **kwargs):
    """torch.distributed process group whose collectives give up after `timeout_s` seconds: a rank that
    died or never joins ends the others' next collective with an error instead of a hang."""
    import torch.distributed as dist
    dist.init_process_group(backend, timeout=timedelta(seconds=timeout_s), **kwargs)


class PeerFailure(RuntimeError):
    """A peer rank did not report a step within the heartbeat timeout."""


class PeerWatch:
    """Host-side heartbeat between steps through a key-value store (the process group's store, or any
    torch.distributed Store): after step s every rank sets ``beat/<rank>`` to s; before launching step
    s + 1 a rank waits up to `timeout_s` for every peer to have reported step s and raises PeerFailure
    naming the ranks that did not.  Nothing here touches a GPU, so a failed peer is noticed before any
    kernel of the next step is in flight."""

    def __init__(self, store, rank: int, world: int, timeout_s: float = 5.0, poll_s: float = 0.01):
        self.store, self.rank, self.world = store, int(rank), int(world)
        self.timeout_s, self.poll_s = float(timeout_s), float(poll_s)

    def beat(self, step: int):
        self.store.set(f"beat/{self.rank}", str(int(step)))

    def _step_of(self, r: int) -> int:
        if not self.store.check([f"beat/{r}"]):
            return -1
        return int(self.store.get(f"beat/{r}"))

    def check(self, step: int):
        deadline = time.monotonic() + self.timeout_s
        while True:
            late = [r for r in range(self.world) if r != self.rank and self._step_of(r) < step]
            if not late:
                return
            if time.monotonic() >= deadline:
                raise PeerFailure(f"ranks {late} did not report step {step} within {self.timeout_s} s")
            time.sleep(self.poll_s)
