"""Training drivers over libgs.

* ``PlainTrainer``  -- the plain form: one scene, one view per optimiser step
  (projection, sort, blend, loss, backward, Adam launched one by one).
* ``BatchedTrainer`` -- the batched form (paper Sec. II trains partitions
  independently; here all partitions and a batch of views per partition are
  one set of units): one gs_train_batch call runs a step of every
  (partition, view) unit, choosing the views on the device from the step
  counter, so the call is captured once in a CUDA graph and every later step
  is a replay with no host work.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

import ctypes as C

from . import _lib, checkpoint
from ._lib import GsTrainBatchDesc, check
from .raster import CHUNK, Adam, Frame, LearningRates, Owned, Units, _alloc_ws, _ptr, _stream, pack_cameras

CAM_BYTES = 96


def psnr(img: torch.Tensor, gt: torch.Tensor, mask: torch.Tensor | None = None) -> float:
    """10 log10(1 / MSE) over the mask pixels (all pixels if no mask) of [3, H, W] images in [0, 1]."""
    d = (img.float().clamp(0, 1) - gt.float()) ** 2
    if mask is not None:
        m = mask.bool()
        if not bool(m.any()):
            return float("nan")
        mse = d[:, m].mean()
    else:
        mse = d.mean()
    return float(10.0 * torch.log10(1.0 / mse.clamp_min(1e-12)))


def split_views(n_views: int, hold_every: int = 8):
    """Every 8th view is held out for evaluation; the rest train."""
    test = list(range(0, n_views, hold_every))
    train = [v for v in range(n_views) if v % hold_every != 0]
    return train, test


class PlainTrainer:
    def __init__(self, params: torch.Tensor, sh_degree: int, cams_dev: torch.Tensor, gt: torch.Tensor,
                 mask: torch.Tensor, train_views, lrs: LearningRates | None = None, extent: float = 1.0,
                 lr_steps: int = 7000, lam: float = 0.2, bg=(1.0, 1.0, 1.0), variant: int = 0, seed: int = 0,
                 capacity_slack: float = 1.5, deterministic: bool = False, chunk: int = CHUNK,
                 densify=None):
        self.params = params
        self.deg = sh_degree
        self.cams = cams_dev
        self._frame_args = dict(variant=variant, deterministic=deterministic, chunk=chunk)
        self.capacity_slack = capacity_slack
        self.gt, self.mask = gt, mask
        self.views = list(train_views)
        self.lam, self.bg = lam, tuple(bg)
        N = params.shape[1]
        H, W = gt.shape[-2], gt.shape[-1]
        self.frame = Frame(N, Units.single(N), W, H, sh_degree, device=params.device, variant=variant,
                           deterministic=deterministic, chunk=chunk)
        self.opt = Adam(params, sh_degree, lrs, extent, lr_steps)
        self.rng = np.random.default_rng(seed)
        self.t = 0
        self.keep_grads = False  # also write the parameter gradient (for inspection)
        self._fit()
        # adaptive density control (3D-GS): a DensifyConfig turns it on
        self.densifier = None
        if densify is not None:
            from .densify import Densifier
            self.densifier = Densifier(N, densify, params.device, seed)
        self.steps_done = 0

    def _fit(self):
        need = max(self.frame.fit_capacity(self.params, self.cam(v))
                   for v in self.views[:: max(1, len(self.views) // 8)])
        self.frame.set_capacity(int(need * self.capacity_slack) + 4096)

    def _densify(self, step: int):
        """Clone / split / prune into new planes; the frame is rebuilt for the new count."""
        d = self.densifier
        counts = d.plan(self.params, step)
        p, m, v = d.apply(self.params, self.opt.m, self.opt.v, self.deg, counts)
        self.params, self.opt.params, self.opt.m, self.opt.v = p, p, m, v
        N = p.shape[1]
        H, W = self.gt.shape[-2], self.gt.shape[-1]
        self.frame = Frame(N, Units.single(N), W, H, self.deg, device=p.device, **self._frame_args)
        self._fit()
        return counts

    def cam(self, v):
        return self.cams[v * CAM_BYTES:(v + 1) * CAM_BYTES]

    def state_dict(self) -> dict:
        """Checkpoint: parameters, optimiser state, step count and the view-order generator (copies).
        In deterministic mode a run resumed from it continues bit for bit like the uninterrupted run."""
        st = {"params": self.params.clone(), "opt": self.opt.state_dict(), "t": self.t,
              "rng": self.rng.bit_generator.state, "steps_done": self.steps_done}
        if hasattr(self, "order"):
            st["order"] = np.array(self.order)
        d = self.densifier
        if d is not None:
            st["densify"] = {"grad_accum": d.grad_accum.clone(), "denom": d.denom.clone(),
                             "max_radius": d.max_radius.clone(), "gen": d.gen.get_state()}
        return st

    def save(self, path: str):
        """Write the checkpoint (state_dict) to a file in the on-disk format of checkpoint.py."""
        checkpoint.save(path, self.state_dict(), self.params.shape[1], self.deg, int(self.opt.step_dev.item()))

    def load(self, path: str):
        """Resume from a file written by save()."""
        self.load_state_dict(checkpoint.load(path, self.params.device)[0])

    def load_state_dict(self, st: dict):
        if st["params"].shape != self.params.shape:  # densification changed the count: new planes, new frame
            p = st["params"].clone()
            self.params, self.opt.params = p, p
            self.opt.m, self.opt.v = torch.zeros_like(p), torch.zeros_like(p)
            N = p.shape[1]
            H, W = self.gt.shape[-2], self.gt.shape[-1]
            self.frame = Frame(N, Units.single(N), W, H, self.deg, device=p.device, **self._frame_args)
            self._fit()
        else:
            self.params.copy_(st["params"])
        self.opt.load_state_dict(st["opt"])
        self.t = int(st["t"])
        self.steps_done = int(st.get("steps_done", 0))
        self.rng.bit_generator.state = st["rng"]
        if "order" in st:
            self.order = np.array(st["order"])
        if "densify" in st and self.densifier is not None:
            d, s = self.densifier, st["densify"]
            d._alloc(self.params.shape[1])
            d.grad_accum.copy_(s["grad_accum"])
            d.denom.copy_(s["denom"])
            d.max_radius.copy_(s["max_radius"])
            d.gen.set_state(s["gen"])

    def next_view(self):
        if self.t % len(self.views) == 0:
            self.order = self.rng.permutation(self.views)
        v = int(self.order[self.t % len(self.views)])
        self.t += 1
        return v

    def step(self, v: int | None = None):
        v = self.next_view() if v is None else v
        fr, cam = self.frame, self.cam(v)
        fr.preprocess(self.params, cam)
        fr.sort()
        fr.render(self.bg)
        fr.loss(self.gt[v:v + 1], self.mask[v:v + 1], self.lam)
        fr.blend_backward(self.bg)
        self.opt.fused_step(fr, cam, self.keep_grads)
        self.steps_done += 1
        d = self.densifier
        if d is not None:
            d.accumulate(fr)
            if d.due(self.steps_done):
                self._densify(self.steps_done)
            if d.reset_due(self.steps_done):
                d.reset_opacity(self.params, self.opt.m, self.opt.v)

    def check(self):
        st = self.frame.read_status()
        if st & 2:  # capacity: grow and continue (lists of the last steps were truncated)
            self.frame.set_capacity(int(self.frame.cap * 1.5))
        return st

    def render(self, v: int):
        self.frame.forward(self.params, self.cam(v), self.bg)
        return self.frame.img[0]

    def evaluate(self, views, gt=None, mask=None) -> float:
        gt = self.gt if gt is None else gt
        mask = self.mask if mask is None else mask
        vals = [psnr(self.render(v), gt[v], mask[v]) for v in views]
        return float(np.nanmean(vals))


class BatchedTrainer:
    """All partitions x ``views_per_step`` views in one graph-captured step.

    params: partition-major planes tensor; part_offsets [n_parts + 1];
    gt [n_parts, V, 3, H, W], mask [n_parts, V, H, W]: each partition's own GT
    and background mask; cams_dev: the V cameras (shared by all partitions)."""

    def __init__(self, params: torch.Tensor, sh_degree: int, part_offsets, cams_dev: torch.Tensor, gt: torch.Tensor,
                 mask: torch.Tensor, train_views, views_per_step: int = 1, lrs: LearningRates | None = None,
                 extent: float = 1.0, lr_steps: int = 7000, lam: float = 0.2, bg=(1.0, 1.0, 1.0), variant: int = 0,
                 use_graph: bool = True, capacity_slack: float = 1.5, deterministic: bool = False,
                 chunk: int = CHUNK, lambda_bg: float = 0.0):
        """lambda_bg > 0 adds the background-opacity penalty (gs_bg_penalty) to every unit's loss."""
        self.params = params
        self.lambda_bg = float(lambda_bg)
        self.deg = sh_degree
        self.off = np.asarray(part_offsets, np.int64)
        self.n_parts = len(self.off) - 1
        self.vps = int(views_per_step)
        self.cams = cams_dev.contiguous()
        self.gt, self.mask = gt.contiguous(), mask.contiguous()
        self.views = list(train_views)
        self.lam, self.bg = lam, tuple(bg)
        self.use_graph = use_graph
        N = params.shape[1]
        H, W = gt.shape[-2], gt.shape[-1]
        dev = params.device
        self.L = _lib.load()
        self.units = Units.partitions(self.off, self.vps)
        U = self.units.n
        self.frame = Frame(N, self.units, W, H, sh_degree, device=dev, variant=variant, deterministic=deterministic,
                           chunk=chunk)
        self.opt = Adam(params, sh_degree, lrs, extent, lr_steps)
        self.cams_step = torch.zeros(U * CAM_BYTES, dtype=torch.uint8, device=dev)
        self.gt_step = torch.zeros((U, 3, H, W), dtype=torch.float32, device=dev)
        self.mask_step = torch.zeros((U, H, W), dtype=torch.uint8, device=dev)
        self.train_views = torch.tensor(self.views, dtype=torch.int32, device=dev)
        self._t_probe = torch.zeros(1, dtype=torch.int32, device=dev)
        self.t = 0
        self.graph = None
        self.keep_grads = False  # also write the parameter gradient (for inspection)
        self.desc = None
        # instance capacity: the largest need over a sweep of the training views
        need = 0
        for t0 in range(0, len(self.views), max(1, len(self.views) // 4)):
            self._load(t0)
            need = max(need, self.frame.fit_capacity(params, self.cams_step))
        self.frame.set_capacity(int(need * capacity_slack) + 4096)

    def view_of(self, t: int, k: int, j: int) -> int:
        """View of unit (partition k, slot j) at step t (staggered across partitions); gs_train_batch applies
        the same rule on the device."""
        return self.views[(t * self.vps + j + k) % len(self.views)]

    def _build_desc(self):
        """The gs_train_batch descriptor: pointers to this trainer's, its frame's and its optimiser's buffers
        (rebuilt when the frame's capacity changes)."""
        fr, opt = self.frame, self.opt
        H, W = fr.H, fr.W
        d = GsTrainBatchDesc()
        d.params, d.adam_m, d.adam_v = self.params.data_ptr(), opt.m.data_ptr(), opt.v.data_ptr()
        d.n_gauss, d.sh_degree, d.views_per_step = self.params.shape[1], self.deg, self.vps
        d.units = C.pointer(self.units.struct)
        d.cam_pool, d.gt_pool, d.mask_pool = self.cams.data_ptr(), self.gt.data_ptr(), self.mask.data_ptr()
        d.train_views, d.n_views, d.n_train = self.train_views.data_ptr(), self.gt.shape[1], len(self.views)
        d.width, d.height, d.lambda_ssim = W, H, float(self.lam)
        d.bg = (C.c_float * 3)(*[float(x) for x in self.bg])
        d.lr_init = opt.lr_init.ctypes.data_as(_lib.c_f32p)
        d.lr_final = opt.lr_final.ctypes.data_as(_lib.c_f32p)
        d.lr_steps, d.beta1, d.beta2, d.eps = opt.lr_steps, opt.b1, opt.b2, opt.eps
        d.d_step = opt.step_dev.data_ptr()
        d.cams_step, d.gt_step, d.mask_step = (self.cams_step.data_ptr(), self.gt_step.data_ptr(),
                                               self.mask_step.data_ptr())
        d.proj = C.pointer(fr.proj)
        d.max_instances, d.sort_ws, d.sort_ws_bytes = fr.cap, fr.sort_ws.data_ptr(), fr.sort_ws.numel()
        d.sorted_vals, d.ranges, d.d_num_instances = (fr.sorted_vals.data_ptr(), fr.ranges.data_ptr(),
                                                      fr.num_instances.data_ptr())
        if fr.use_masks:
            fr.sched.walk_whole_lists = 1 if fr.walk_whole_lists else 0
            d.sched = C.pointer(fr.sched)
        d.img, d.final_T, d.n_contrib = fr.img.data_ptr(), fr.final_T.data_ptr(), fr.n_contrib.data_ptr()
        d.loss_ws, d.loss_ws_bytes = fr.loss_ws.data_ptr(), fr.loss_ws.numel()
        d.d_loss, d.dL_dimg = fr.loss_val.data_ptr(), fr.dimg.data_ptr()
        d.g2d = C.pointer(fr.g2d)
        d.grads = fr.grads.data_ptr() if self.keep_grads else None
        d.variant = fr.variant
        d.sparse_adam = int(opt.sparse)
        if self.lambda_bg > 0.0:
            if fr.dL_dT is None:
                fr.dL_dT = torch.zeros((self.units.n, H, W), dtype=torch.float32, device=self.params.device)
                fr.bg_ws = _alloc_ws(self.L.gs_bg_penalty_workspace_size(self.units.n), self.params.device)
            d.lambda_bg, d.bg_ws, d.bg_ws_bytes = self.lambda_bg, fr.bg_ws.data_ptr(), fr.bg_ws.numel()
            d.dL_dT = fr.dL_dT.data_ptr()
        self.desc = d
        self._desc_key = (fr.cap, self.keep_grads, fr.use_masks, fr.walk_whole_lists, opt.sparse)

    def _load(self, t: int):
        """The step buffers of step t (gs_gather_views on the device), for inspection and capacity sizing."""
        if self.desc is None:
            self._build_desc()
        self._t_probe.fill_(int(t))
        check(self.L.gs_gather_views(C.byref(self.desc), _ptr(self._t_probe), _stream()), "gs_gather_views")

    def _chain(self):
        fr = self.frame
        if self.desc is None or self._desc_key != (fr.cap, self.keep_grads, fr.use_masks, fr.walk_whole_lists,
                                                   self.opt.sparse):
            self._build_desc()
        check(self.L.gs_train_batch(C.byref(self.desc), _ptr(fr.status), _stream()), "gs_train_batch")

    def capture(self):
        """Run step t eagerly (on a side stream, so lazy initialisation happens outside the capture), then
        record the whole training step (one gs_train_batch call) as a CUDA graph for the following steps."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self._chain()
        torch.cuda.current_stream().wait_stream(s)
        self.t += 1
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._chain()
        self.graph = g

    def step(self):
        """One training step of every unit; its views follow from the device step counter."""
        if self.use_graph and self.graph is None:
            self.capture()
            return
        if self.use_graph:
            self.graph.replay()
        else:
            self._chain()
        self.t += 1

    def state_dict(self) -> dict:
        """Checkpoint: parameters, optimiser state and step count (copies); views follow from the step."""
        return {"params": self.params.clone(), "opt": self.opt.state_dict(), "t": self.t}

    def save(self, path: str):
        """Write the checkpoint (state_dict) to a file in the on-disk format of checkpoint.py."""
        checkpoint.save(path, self.state_dict(), self.params.shape[1], self.deg, int(self.opt.step_dev.item()))

    def load(self, path: str):
        """Resume from a file written by save()."""
        self.load_state_dict(checkpoint.load(path, self.params.device)[0])

    def load_state_dict(self, st: dict):
        """Restore a checkpoint in place (the captured graph reads the same buffers, so it stays valid)."""
        self.params.copy_(st["params"])
        self.opt.load_state_dict(st["opt"])
        self.t = int(st["t"])

    def check(self):
        st = self.frame.read_status()
        if st & 2:
            self.frame.set_capacity(int(self.frame.cap * 1.5))
            self.graph = None  # buffers changed: capture again
        return st

    def merged(self, part) -> Owned:
        return Owned(self.off, part.boxes, part.closed_hi)

    def merge_render(self, owned: Owned, cam_dev: torch.Tensor, width: int, height: int, frame: Frame | None = None):
        N = self.params.shape[1]
        fr = frame or Frame(N, Units.single(N), width, height, self.deg, device=self.params.device,
                            with_backward=False, with_loss=False)
        fr.fit_capacity(self.params, cam_dev, owned)
        fr.merge_render(self.params, cam_dev, self.bg, owned)
        return fr.img[0], fr
