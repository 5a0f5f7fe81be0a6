"""Plain form vs batched + learned-init form, PSNR against wall-clock time.

1. Train the plain form (plain kNN initialisation, one view per step) on a
   source scene; its converged splats are the MLP's regression targets.
2. Train the MLP (gs_mlp_train_step) on the source scene's points.
3. On a new target scene, run (a) the plain form and (b) the learned
   initialisation followed by the graph-captured batched trainer, evaluating
   held-out-view PSNR at checkpoints; report how long (b) takes to reach the
   PSNR (a) reaches, within a tolerance.

Times exclude evaluation renders (the clock is stopped around them).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import init as gi
from .raster import LearningRates, pack_params
from .train import BatchedTrainer, PlainTrainer, psnr, split_views


@dataclass
class History:
    steps: list = field(default_factory=list)
    seconds: list = field(default_factory=list)
    psnr: list = field(default_factory=list)

    def add(self, s, t, p):
        self.steps.append(int(s))
        self.seconds.append(float(t))
        self.psnr.append(float(p))

    def time_to(self, target: float):
        for s, t, p in zip(self.steps, self.seconds, self.psnr):
            if p >= target:
                return s, t
        return None, None


def _points(scene, device):
    return (torch.from_numpy(scene.pts).to(device).contiguous(), torch.from_numpy(scene.nrm).to(device).contiguous())


def evaluate(render, scene, views) -> float:
    vals = [psnr(render(v), scene.gt[v], scene.mask[v]) for v in views]
    return float(np.nanmean(vals))


def run_plain(scene, steps: int, eval_every: int, device="cuda", lrs: LearningRates | None = None):
    """Plain form: plain kNN init, one view per optimiser step, launches one by one."""
    train_v, test_v = split_views(len(scene.cams))
    P, Nn = _points(scene, device)
    params = pack_params(scene.init, scene.sh_degree, device)
    gi.init_gaussians(params, P)  # plain form: mean 3-NN distance scale, identity rotation, opacity 0.1
    tr = PlainTrainer(params, scene.sh_degree, scene.cams_dev, scene.gt, scene.mask, train_v, lrs=lrs,
                      lr_steps=steps)
    h = History()
    h.add(0, 0.0, tr.evaluate(test_v))
    clock = 0.0
    for s0 in range(0, steps, eval_every):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(min(eval_every, steps - s0)):
            tr.step()
        torch.cuda.synchronize()
        clock += time.perf_counter() - t0
        tr.check()
        h.add(s0 + eval_every, clock, tr.evaluate(test_v))
    return h, params


def fit_mlp(scene, trained_params, steps: int = 600, lr: float = 2e-3, seed: int = 0, device="cuda"):
    """Train the initialiser MLP on one scene's points against its converged splats."""
    P, Nn = _points(scene, device)
    idx, dist = gi.knn(P, 16)
    targets = gi.targets_from_params(trained_params, dist)
    w = gi.init_weights(seed, device)
    tr = gi.MLPTrainer(w, lr=lr)
    losses = []
    for k in range(steps):
        l = tr.step(P, Nn, idx, dist, targets)
        if k % 50 == 0 or k == steps - 1:
            losses.append(float(l.item()))
    return w, losses


def run_learned_batched(scene, weights, steps: int, eval_every: int, views_per_step: int = 2, variant: int = 0,
                        device="cuda", lrs: LearningRates | None = None, stop_at: float | None = None):
    """Learned initialisation, then the graph-captured batched trainer (one partition, a batch of views)."""
    train_v, test_v = split_views(len(scene.cams))
    P, Nn = _points(scene, device)
    params = pack_params(scene.init, scene.sh_degree, device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    idx, dist = gi.knn(P, 16)
    gi.init_gaussians(params, P, Nn, weights, idx, dist)
    torch.cuda.synchronize()
    clock = time.perf_counter() - t0  # the initialiser's cost counts against this form
    off = np.array([0, scene.n], np.int64)
    tr = BatchedTrainer(params, scene.sh_degree, off, scene.cams_dev, scene.gt[None], scene.mask[None], train_v,
                        views_per_step=views_per_step, lrs=lrs, lr_steps=steps, variant=variant)
    from .raster import Frame, Units
    fr = Frame(scene.n, Units.single(scene.n), scene.width, scene.height, scene.sh_degree, device=device,
               with_backward=False, with_loss=False)
    fr.set_capacity(tr.frame.cap)

    def render(v):
        fr.forward(params, scene.cam(v), scene.bg)
        return fr.img[0]

    h = History()
    h.add(0, clock, evaluate(render, scene, test_v))
    for s0 in range(0, steps, eval_every):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(min(eval_every, steps - s0)):
            tr.step()
        torch.cuda.synchronize()
        clock += time.perf_counter() - t0
        tr.check()
        h.add(s0 + eval_every, clock, evaluate(render, scene, test_v))
        if stop_at is not None and h.psnr[-1] >= stop_at:
            break
    return h, params
