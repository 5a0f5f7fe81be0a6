"""Spatial partitioning with ghost cells (paper Sec. II, "Data Partitioning").

The domain is cut into n slabs along x.  Partition k owns the half-open slab
[x_k, x_{k+1}) (the last one closed) and additionally receives the points of a
ghost layer of width ghost * slab_width on each interior side, so that splats
near a cut are trained in both neighbours and the merged render shows no gap
(Sec. III-A, Fig. 2).  For the merge (Sec. II, "Global Reconstruction") a
partition keeps only the Gaussians whose trained mean lies in its owned slab.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BIG = 1e30


@dataclass
class Partition:
    members: list            # per partition: indices into the source point set (owned + ghost)
    offsets: np.ndarray      # [n + 1] prefix offsets of the partition-major concatenation
    boxes: np.ndarray        # [n, 6] owned boxes (xmin, ymin, zmin, xmax, ymax, zmax)
    closed_hi: np.ndarray    # [n] bit a set: upper bound of axis a is closed
    edges: np.ndarray        # [n + 1] slab edges along x

    @property
    def n(self) -> int:
        return len(self.members)

    @property
    def order(self) -> np.ndarray:
        """Source index of every entry of the partition-major concatenation."""
        return np.concatenate(self.members) if self.members else np.zeros(0, np.int64)

    def sizes(self):
        return np.diff(self.offsets)


def slab_partition(points, n_parts: int = 8, ghost: float = 0.05, lo: float = 0.0, hi: float = 1.0) -> Partition:
    x = np.asarray(points)[:, 0].astype(np.float64)
    edges = np.linspace(lo, hi, n_parts + 1)
    w = (hi - lo) / n_parts
    members = []
    for k in range(n_parts):
        a = edges[k] - (ghost * w if k > 0 else 0.0)
        b = edges[k + 1] + (ghost * w if k < n_parts - 1 else 0.0)
        if k == n_parts - 1:
            sel = (x >= a) & (x <= b)
        else:
            sel = (x >= a) & (x < b)
        members.append(np.nonzero(sel)[0].astype(np.int64))
    offsets = np.concatenate([[0], np.cumsum([len(m) for m in members])]).astype(np.int64)
    boxes = np.zeros((n_parts, 6), np.float32)
    boxes[:, 0] = edges[:-1]
    boxes[:, 3] = edges[1:]
    boxes[:, 1] = boxes[:, 2] = -BIG
    boxes[:, 4] = boxes[:, 5] = BIG
    closed = np.full(n_parts, 0b110, np.int32)
    closed[-1] |= 0b001
    return Partition(members=members, offsets=offsets, boxes=boxes, closed_hi=closed, edges=edges)


def owned_mask(means, part: Partition) -> np.ndarray:
    """Host reference of the ghost filter for a partition-major array of means."""
    means = np.asarray(means, np.float64)
    keep = np.zeros(len(means), bool)
    for k in range(part.n):
        s, e = part.offsets[k], part.offsets[k + 1]
        b = part.boxes[k].astype(np.float64)
        m = means[s:e]
        ok = np.ones(e - s, bool)
        for a in range(3):
            hi_ok = (m[:, a] <= b[3 + a]) if (part.closed_hi[k] >> a) & 1 else (m[:, a] < b[3 + a])
            ok &= (m[:, a] >= b[a]) & hi_ok
        keep[s:e] = ok
    return keep
