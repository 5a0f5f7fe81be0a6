"""Initialisation of the Gaussians from isosurface points (plain and learned).

Plain form: isotropic scale from the mean distance to the 3 nearest
neighbours, identity rotation, opacity 0.1.  Learned form: a small MLP (libgs
gs_mlp_*) predicts scale offsets, rotation and opacity from the 16-neighbour
geometry; it is trained on converged splats produced by the method itself,
and the plain form stays both the fallback and the reference it must beat.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _lib
from ._lib import check
from .raster import _ptr, _stream

N_PARAMS = 11912
LOGIT_01 = math.log(0.1 / 0.9)


def grid_for(points: torch.Tensor, k: int):
    """Uniform grid over the points' bounding box with cells about the size of the k-NN radius of a
    surface sample: density lam = n / (product of the two largest extents), h = sqrt(k / (pi lam))."""
    lo = points.min(dim=0).values.double().cpu().numpy()
    hi = points.max(dim=0).values.double().cpu().numpy()
    ext = np.maximum(hi - lo, 1e-6)
    n = max(points.shape[0], 1)
    e = np.sort(ext)
    lam = n / (e[1] * e[2])
    h = math.sqrt(k / (math.pi * lam))
    h = max(h, float(ext.max()) / 4096.0)
    dims = np.maximum(np.ceil(ext / h).astype(np.int64) + 1, 1)
    while int(np.prod(dims)) > (1 << 26):
        h *= 1.25
        dims = np.maximum(np.ceil(ext / h).astype(np.int64) + 1, 1)
    lo = lo - 0.5 * h
    return lo.astype(np.float32), float(h), dims.astype(np.int32)


def knn(points: torch.Tensor, k: int):
    """Exact k nearest neighbours of [n, 3] float32 device points: (idx int32 [n, k], dist float32 [n, k])."""
    L = _lib.load()
    points = points.contiguous()
    n = points.shape[0]
    lo, h, dims = grid_for(points, k)
    ws_bytes = L.gs_knn_workspace_size(n, dims.ctypes.data_as(_lib.c_i32p))
    ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=points.device)
    idx = torch.empty((n, k), dtype=torch.int32, device=points.device)
    dist = torch.empty((n, k), dtype=torch.float32, device=points.device)
    check(L.gs_knn(_ptr(points), n, k, lo.ctypes.data_as(_lib.c_f32p), h, dims.ctypes.data_as(_lib.c_i32p),
                   _ptr(ws), ws_bytes, _ptr(idx), _ptr(dist), _stream()), "gs_knn")
    return idx, dist


def init_gaussians(params: torch.Tensor, points: torch.Tensor, normals: torch.Tensor | None = None,
                   weights: torch.Tensor | None = None, knn_idx=None, knn_dist=None, logit_default=LOGIT_01):
    """Write means, scales, rotations and opacities of the first n Gaussians of a planes tensor.
    weights None: plain form (needs 3 neighbours); else the learned form (16 neighbours)."""
    L = _lib.load()
    n = points.shape[0]
    kk = 3 if weights is None else 16
    if knn_dist is None or knn_dist.shape[1] < kk or (weights is not None and knn_dist.shape[1] != 16):
        knn_idx, knn_dist = knn(points, kk)
    check(L.gs_init_gaussians(_ptr(points.contiguous()), _ptr(normals) if normals is not None else None,
                              _ptr(knn_idx) if knn_idx is not None else None, _ptr(knn_dist.contiguous()),
                              knn_dist.shape[1], n, _ptr(weights) if weights is not None else None,
                              float(logit_default), _ptr(params), params.shape[1], _stream()), "gs_init_gaussians")
    return params


def init_weights(seed: int = 0, device="cuda") -> torch.Tensor:
    """He-initialised weights with a zero last layer (so an untrained network gives the plain form's scale,
    and identity rotation through the bias)."""
    g = np.random.default_rng(seed)
    w = np.zeros(N_PARAMS, np.float32)
    o = 0
    W1 = g.standard_normal((112, 64)) * math.sqrt(2.0 / 99.0)
    w[o:o + 7168] = W1.reshape(-1); o += 7168
    o += 64
    W2 = g.standard_normal((64, 64)) * math.sqrt(2.0 / 64.0)
    w[o:o + 4096] = W2.reshape(-1); o += 4096
    o += 64
    o += 512  # W3 = 0
    b3 = np.array([0, 0, 0, 1, 0, 0, 0, LOGIT_01], np.float32)
    w[o:o + 8] = b3
    return torch.from_numpy(w).to(device)


def targets_from_params(trained: torch.Tensor, knn_dist: torch.Tensor) -> torch.Tensor:
    """Regression targets [n, 8] from converged planes: log-scale minus log(d3), the rotation normalised with
    w >= 0 (q and -q are the same rotation), the logit opacity."""
    n = knn_dist.shape[0]
    d3 = knn_dist[:, :3].mean(dim=1).clamp_min(1e-7)
    ls = trained[1, :n, :3] - torch.log(d3)[:, None]
    q = trained[2, :n]
    q = q / q.norm(dim=1, keepdim=True).clamp_min(1e-12)
    q = torch.where(q[:, :1] < 0, -q, q)
    lo = trained[1, :n, 3:4]
    return torch.cat([ls, q, lo], dim=1).contiguous()


class MLPTrainer:
    """Adam on the MLP weights with gs_mlp_train_step (full batch)."""

    def __init__(self, weights: torch.Tensor, lr: float = 1e-3):
        self.L = _lib.load()
        self.w = weights
        self.grad = torch.zeros_like(weights)
        self.m = torch.zeros_like(weights)
        self.v = torch.zeros_like(weights)
        self.step_dev = torch.zeros(1, dtype=torch.int32, device=weights.device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=weights.device)
        self.lr = lr

    def step(self, points, normals, knn_idx, knn_dist, targets, n: int | None = None):
        """One Adam step on the first n points (all by default; neighbour indices may point anywhere in
        ``points``)."""
        n = points.shape[0] if n is None else int(n)
        check(self.L.gs_mlp_train_step(_ptr(points), _ptr(normals), _ptr(knn_idx), _ptr(knn_dist), _ptr(targets), n,
                                       _ptr(self.w), _ptr(self.grad), _ptr(self.m), _ptr(self.v), float(self.lr),
                                       _ptr(self.step_dev), _ptr(self.loss), _stream()), "gs_mlp_train_step")
        check(self.L.gs_step_advance(_ptr(self.step_dev), _stream()), "gs_step_advance")
        return self.loss


def mlp_forward(weights, points, normals, knn_idx, knn_dist) -> torch.Tensor:
    L = _lib.load()
    n = points.shape[0]
    out = torch.empty((n, 8), dtype=torch.float32, device=points.device)
    check(L.gs_mlp_forward(_ptr(points), _ptr(normals), _ptr(knn_idx), _ptr(knn_dist), n, _ptr(weights), _ptr(out),
                           _stream()), "gs_mlp_forward")
    return out


def mlp_features(points, normals, knn_idx, knn_dist) -> torch.Tensor:
    """bf16 bit patterns [n, 112] of the network inputs (as int16 tensor)."""
    L = _lib.load()
    n = points.shape[0]
    out = torch.empty((n, 112), dtype=torch.int16, device=points.device)
    check(L.gs_mlp_features(_ptr(points), _ptr(normals), _ptr(knn_idx), _ptr(knn_dist), n, _ptr(out), _stream()),
          "gs_mlp_features")
    return out
