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


def subset_first(P, Nn, idx, dist, targets, seed: int):
    """The cloud in a seeded random order, its neighbour indices renumbered to match: any first n rows are
    then a random subset whose neighbours (anywhere in the cloud) are the same points as before.  The MLP
    train step takes its own points from rows 0 .. n - 1."""
    n = P.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(n, generator=g).to(P.device)
    inv = torch.empty_like(perm)
    inv[perm] = torch.arange(n, device=P.device)
    return (P[perm].contiguous(), Nn[perm].contiguous(), inv[idx[perm].long()].to(idx.dtype).contiguous(),
            dist[perm].contiguous(), targets[perm].contiguous())


def fit_mlp(scene, trained_params, steps: int = 600, lr: float = 2e-3, seed: int = 0, device="cuda",
            fit_points: int | None = None):
    """Train the initialiser MLP on one scene's points against its converged splats.  fit_points: train on
    a seeded random subset of that many points (their neighbours still come from the whole cloud); all
    points when None or not smaller than the scene."""
    P, Nn = _points(scene, device)
    idx, dist = gi.knn(P, 16)
    targets = gi.targets_from_params(trained_params, dist)
    n = P.shape[0]
    n_fit = n
    if fit_points is not None and fit_points < n:
        P, Nn, idx, dist, targets = subset_first(P, Nn, idx, dist, targets, seed)
        n_fit = int(fit_points)
    w = gi.init_weights(seed, device)
    tr = gi.MLPTrainer(w, lr=lr)
    losses = []
    for k in range(steps):
        l = tr.step(P, Nn, idx, dist, targets, n_fit)
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


def seam_band(scene, delta: float, device="cuda"):
    """Per view, the pixels whose visible surface lies within `delta` (in x) of an interior slab boundary:
    the ground-truth surfels rendered with their x coordinate as colour (opaque, so a covered pixel shows
    the x of its front surface), compared with the partition edges.  Returns bool [V, H, W]."""
    from .workload import gt_surfels, render_gt
    pts = scene.pts
    nrm = scene.nrm
    xcol = np.repeat(pts[:, :1], 3, axis=1).astype(np.float32)
    ximg, cover = render_gt(gt_surfels(pts, nrm, xcol, scene.spacing), scene.cams, 0, (-1.0, -1.0, -1.0), device,
                            max_instances=max(8 * len(pts), 1 << 20))
    edges = torch.tensor(np.asarray(scene.part.edges[1:-1], np.float32), device=device)
    d = (ximg[:, 0, :, :, None] - edges).abs().amin(-1)
    return (d < delta) & cover.bool()


def ghost_ablation(slab_counts, n_modes: int, n_views: int, W: int, H: int, steps: int, n_parts: int = 4,
                   ghost: float = 0.05, sh_degree: int = 1, delta: float = 0.01, device="cuda",
                   init_scale: float = 1.0, lambda_bg: float = 0.0):
    """Ghost cells and masks on and off (Sec. II): each configuration trains every partition on its own
    GT (graph-captured batched trainer, one view per partition per step), merges with the ghost filter and
    is scored on held-out views against the whole scene's GT: PSNR over the covered pixels and over the
    seam band (pixels whose surface lies within `delta` of a slab boundary).  lambda_bg > 0 adds the mask
    variant "mask=on+bg": the masked loss plus the background-opacity penalty of that weight (the mean
    rendered opacity over the pixels outside the mask, gs_bg_penalty)."""
    from .raster import Frame, Owned, Units
    from .workload import partitioned_scene
    out = {}
    band = None
    for use_ghost in (True, False):
        ps = partitioned_scene(slab_counts, n_modes, n_views, W, H, n_parts=n_parts,
                               ghost=ghost if use_ghost else 0.0, sh_degree=sh_degree, device=device,
                               init_scale=init_scale)
        if band is None:
            band = seam_band(ps, delta, device)
        train_v, test_v = split_views(n_views)
        modes = [("on", True, 0.0), ("off", False, 0.0)] + ([("on+bg", True, lambda_bg)] if lambda_bg > 0 else [])
        for mode, use_mask, lam_bg in modes:
            masks = ps.mask if use_mask else torch.ones_like(ps.mask)
            params = pack_params(ps.init, sh_degree, device)
            tr = BatchedTrainer(params, sh_degree, ps.offsets, ps.cams_dev, ps.gt, masks, train_v, views_per_step=1,
                                lr_steps=steps, lambda_bg=lam_bg)
            t0 = time.perf_counter()
            for _ in range(steps):
                tr.step()
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            tr.check()
            owned = Owned(ps.part.offsets, ps.part.boxes, ps.part.closed_hi)
            N = params.shape[1]
            fr = Frame(N, Units.single(N), W, H, sh_degree, device=device, with_backward=False, with_loss=False)
            fr.walk_whole_lists = True
            all_p, band_p = [], []
            for v in test_v:
                cam = ps.cams_dev[v * 96:(v + 1) * 96]
                fr.fit_capacity(params, cam, owned)
                img = fr.merge_render(params, cam, ps.bg, owned)[0]
                all_p.append(psnr(img, ps.gt_full[v], ps.mask_full[v]))
                band_p.append(psnr(img, ps.gt_full[v], band[v]))
            key = f"ghost={'on' if use_ghost else 'off'},mask={mode}"
            out[key] = {"psnr_covered": round(float(np.nanmean(all_p)), 3),
                        "psnr_seam_band": round(float(np.nanmean(band_p)), 3),
                        "train_seconds": round(secs, 3),
                        "gaussians_with_ghosts": int(N)}
            del tr, fr, params
            torch.cuda.empty_cache()
    out["seam_band_fraction_of_covered"] = round(float(band.float().sum() / ps.mask_full.float().sum()), 4)
    return out
