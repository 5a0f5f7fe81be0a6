"""Buffers, packing and the autograd wrapper around libgs.

PyTorch provides device memory, the stream and the autograd hook; every step
of the rasterizer runs in libgs kernels (see include/gs.h).
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import GsCamera, GsGrad2d, GsOwned, GsProj, GsSchedule, GsUnits, check

CHUNK = 1024  # list entries per backward chunk job

TILE = 16


def param_planes(sh_degree: int) -> int:
    return 3 + (3 * (sh_degree + 1) ** 2 + 3) // 4


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- packing
def pack_params(g: dict, sh_degree: int, device="cuda") -> torch.Tensor:
    """Gaussian dict (means, log_scales, quats, logit_opacity, sh[N, (d+1)^2, 3]) -> planes [n_planes, N, 4] fp32."""
    n = np.asarray(g["means"]).shape[0]
    npl = param_planes(sh_degree)
    out = np.zeros((npl, n, 4), np.float32)
    out[0, :, :3] = g["means"]
    out[1, :, :3] = g["log_scales"]
    out[1, :, 3] = g["logit_opacity"]
    out[2] = g["quats"]
    nc = (sh_degree + 1) ** 2
    sh = np.asarray(g["sh"], np.float32).reshape(n, -1)[:, : 3 * nc]
    flat = np.zeros((n, (npl - 3) * 4), np.float32)
    flat[:, : 3 * nc] = sh
    out[3:] = flat.reshape(n, npl - 3, 4).transpose(1, 0, 2)
    return torch.from_numpy(out).to(device)


def unpack_params(t: torch.Tensor, sh_degree: int) -> dict:
    a = t.detach().cpu().numpy()
    n = a.shape[1]
    nc = (sh_degree + 1) ** 2
    sh = a[3:].transpose(1, 0, 2).reshape(n, -1)[:, : 3 * nc].reshape(n, nc, 3)
    return dict(means=a[0, :, :3].copy(), log_scales=a[1, :, :3].copy(), logit_opacity=a[1, :, 3].copy(),
                quats=a[2].copy(), sh=sh.copy())


def unpack_grads(t: torch.Tensor, sh_degree: int) -> np.ndarray:
    """Planes -> [N, n_params] in the order mean, log-scale, quat, logit, SH."""
    d = unpack_params(t, sh_degree)
    n = d["means"].shape[0]
    return np.concatenate([d["means"], d["log_scales"], d["quats"], d["logit_opacity"][:, None],
                           d["sh"].reshape(n, -1)], axis=1)


CAMERA_DTYPE = np.dtype([("viewmat", np.float32, 12), ("fx", np.float32), ("fy", np.float32), ("cx", np.float32),
                         ("cy", np.float32), ("tan_fovx", np.float32), ("tan_fovy", np.float32),
                         ("campos", np.float32, 3), ("znear", np.float32), ("width", np.int32),
                         ("height", np.int32)])
assert CAMERA_DTYPE.itemsize == C.sizeof(GsCamera)


def pack_cameras(cams, device="cuda") -> torch.Tensor:
    """synth.Cameras -> device byte tensor holding gs_camera structs."""
    n = len(cams)
    a = np.zeros(n, CAMERA_DTYPE)
    a["viewmat"] = np.asarray(cams.viewmat, np.float32).reshape(n, 12)
    for f in ("fx", "fy", "cx", "cy", "tan_fovx", "tan_fovy"):
        a[f] = getattr(cams, f)
    a["campos"] = cams.campos
    a["znear"] = cams.znear
    a["width"] = cams.width
    a["height"] = cams.height
    return torch.from_numpy(a.view(np.uint8).copy()).to(device)


class Units:
    """Host-side unit table: unit u renders Gaussians [begin[u], begin[u] + count[u])."""

    def __init__(self, begin, count):
        self.begin = np.ascontiguousarray(begin, dtype=np.int64)
        self.count = np.ascontiguousarray(count, dtype=np.int64)
        assert self.begin.shape == self.count.shape and self.begin.ndim == 1
        self.n = int(self.begin.shape[0])
        self.proj_base = np.concatenate([[0], np.cumsum(self.count)]).astype(np.int64)
        self.struct = GsUnits(self.n, self.begin.ctypes.data_as(_lib.c_i64p), self.count.ctypes.data_as(_lib.c_i64p))

    @property
    def n_proj(self) -> int:
        return int(self.proj_base[-1])

    @staticmethod
    def single(n_gauss: int, n_views: int = 1) -> "Units":
        return Units([0] * n_views, [n_gauss] * n_views)

    @staticmethod
    def partitions(part_offsets, n_views: int) -> "Units":
        """Unit k * n_views + v = (partition k, view v)."""
        off = np.asarray(part_offsets, np.int64)
        b, c = [], []
        for k in range(len(off) - 1):
            for _ in range(n_views):
                b.append(off[k])
                c.append(off[k + 1] - off[k])
        return Units(b, c)


class Owned:
    """Ghost filter for the merged render."""

    def __init__(self, part_offsets, boxes, closed_hi):
        self.off = np.ascontiguousarray(part_offsets, np.int64)
        self.boxes = np.ascontiguousarray(boxes, np.float32).reshape(-1, 6)
        self.closed = np.ascontiguousarray(closed_hi, np.int32)
        self.struct = GsOwned(int(len(self.off) - 1), self.off.ctypes.data_as(_lib.c_i64p),
                              self.boxes.ctypes.data_as(_lib.c_f32p), self.closed.ctypes.data_as(_lib.c_i32p))


def _alloc_ws(nbytes: int, device) -> torch.Tensor:
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


class Frame:
    """All device buffers of one rasterizer configuration (N Gaussians, a unit table, W x H)."""

    def __init__(self, n_gauss: int, units: Units, width: int, height: int, sh_degree: int, device="cuda",
                 max_instances: int | None = None, with_backward: bool = True, with_loss: bool = True,
                 variant: int = 0, chunk: int = CHUNK, deterministic: bool = False):
        self.L = _lib.load()
        self.variant = int(variant)
        self.chunk = int(chunk)
        self.use_masks = True  # per-instance block masks from the sort drive the blend kernels' culling
        # forward: chunks of a list composited in parallel and combined (False), or one walk per list
        # that stops at its pixels' last stop (True: renders of opaque, trained scenes)
        self.walk_whole_lists = False
        self.device = torch.device(device)
        self.N = int(n_gauss)
        self.units = units
        self.W, self.H = int(width), int(height)
        self.deg = int(sh_degree)
        self.planes = param_planes(self.deg)
        P = units.n_proj
        self.P = P
        self.TX, self.TY = (self.W + TILE - 1) // TILE, (self.H + TILE - 1) // TILE
        self.n_tiles = self.TX * self.TY
        U = units.n
        f32 = dict(dtype=torch.float32, device=self.device)
        # pixel-space means as float pairs (x, y, x_lo, y_lo); xy64() gives x + x_lo, y + y_lo
        self.xy = torch.zeros((max(P, 1), 4), **f32)
        self.conic_op = torch.zeros((max(P, 1), 4), **f32)
        self.rgb = torch.zeros((max(P, 1), 4), **f32)
        self.depth = torch.zeros(max(P, 1), **f32)
        self.radius = torch.zeros(max(P, 1), dtype=torch.int32, device=self.device)
        self.tiles = torch.zeros(max(P, 1), dtype=torch.int32, device=self.device)
        self.proj = GsProj(self.xy.data_ptr(), self.conic_op.data_ptr(), self.rgb.data_ptr(), self.depth.data_ptr(),
                           self.radius.data_ptr(), self.tiles.data_ptr())
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.set_capacity(max_instances if max_instances is not None else max(4 * P, 1024))
        self.ranges = torch.zeros((U * self.n_tiles, 2), dtype=torch.int32, device=self.device)
        self.img = torch.zeros((U, 3, self.H, self.W), **f32)
        self.final_T = torch.zeros((U, self.H, self.W), **f32)
        self.n_contrib = torch.zeros((U, self.H, self.W), dtype=torch.int32, device=self.device)
        if with_loss:
            self.loss_ws = _alloc_ws(self.L.gs_loss_workspace_size(U, self.W, self.H), self.device)
            self.loss_val = torch.zeros(1, **f32)
            self.dimg = torch.zeros((U, 3, self.H, self.W), **f32)
        self.dL_dT = None  # dpenalty/dT_final of the background-opacity penalty (made by bg_penalty)
        if with_backward:
            self.dxy = torch.zeros((max(P, 1), 2), **f32)
            self.dco = torch.zeros((max(P, 1), 4), **f32)
            self.drgb = torch.zeros((max(P, 1), 4), **f32)
            # deterministic: screen-space gradients accumulate as int64 fixed point (bitwise reproducible)
            self.fixed = torch.zeros((max(P, 1), 9), dtype=torch.int64, device=self.device) if deterministic else None
            self.g2d = GsGrad2d(self.dxy.data_ptr(), self.dco.data_ptr(), self.drgb.data_ptr(),
                                self.fixed.data_ptr() if deterministic else None)
            self.grads = torch.zeros((self.planes, max(self.N, 1), 4), **f32)

    def _sched(self):
        if not self.use_masks:
            return None
        self.sched.walk_whole_lists = 1 if self.walk_whole_lists else 0
        return C.byref(self.sched)

    def set_capacity(self, max_instances: int):
        self.cap = int(max_instances)
        ws = self.L.gs_bin_sort_workspace_size(self.P, self.cap)
        self.sort_ws = _alloc_ws(ws, self.device)
        self.sorted_vals = torch.zeros(max(self.cap, 1), dtype=torch.int32, device=self.device)
        self.block_masks = torch.zeros(max(self.cap, 1), dtype=torch.int16, device=self.device)
        mj, mc = C.c_int64(), C.c_int64()
        check(self.L.gs_schedule_sizes(self.units.n, self.W, self.H, self.cap, self.chunk, C.byref(mj), C.byref(mc)),
              "gs_schedule_sizes")
        nt = self.units.n * self.n_tiles
        self.tile_order = torch.zeros(nt, dtype=torch.int32, device=self.device)
        self.job_base = torch.zeros(nt + 1, dtype=torch.int32, device=self.device)
        self.jobs = torch.zeros(2 * mj.value, dtype=torch.int32, device=self.device)
        self.checkpoints = torch.zeros((mc.value, 256, 4), dtype=torch.float32, device=self.device)
        self.chunk_last = torch.zeros((mc.value, 256), dtype=torch.int32, device=self.device)
        self.stop_queue = torch.zeros(8 * mj.value + 1, dtype=torch.int32, device=self.device)
        self.sched = GsSchedule(self.tile_order.data_ptr(), self.block_masks.data_ptr(), self.job_base.data_ptr(),
                                self.jobs.data_ptr(), self.checkpoints.data_ptr(), self.chunk_last.data_ptr(),
                                self.stop_queue.data_ptr(), mj.value, mc.value, self.chunk)
        self.num_instances = torch.zeros(1, dtype=torch.int32, device=self.device)

    # -- steps
    def preprocess(self, params: torch.Tensor, cams_dev: torch.Tensor, owned: Owned | None = None):
        assert params.is_contiguous() and params.shape[0] == self.planes and params.shape[1] == self.N
        check(self.L.gs_preprocess(_ptr(params), self.N, self.deg, C.byref(self.units.struct), _ptr(cams_dev),
                                   self.W, self.H, C.byref(owned.struct) if owned is not None else None,
                                   C.byref(self.proj), _ptr(self.status), _stream()), "gs_preprocess")

    sort_design = "depth_first"

    def sort(self, design: str = None):
        """gs_bin_sort (records sorted by depth, then their instances binned), gs_bin_sort_global (one radix
        sort of all instance keys) or gs_bin_sort_bucketed (per-list sorts); all three give the same lists.
        design: "depth_first", "global" or "bucketed" (default: the frame's sort_design)."""
        design = design or self.sort_design
        fn = {"depth_first": self.L.gs_bin_sort, "global": self.L.gs_bin_sort_global,
              "bucketed": self.L.gs_bin_sort_bucketed}[design]
        check(fn(C.byref(self.proj), C.byref(self.units.struct), self.W, self.H, self.cap, _ptr(self.sort_ws),
                 self.sort_ws.numel(), _ptr(self.sorted_vals), _ptr(self.ranges), _ptr(self.num_instances),
                 self._sched(), _ptr(self.status), _stream()), "gs_bin_sort")

    def render(self, bg):
        bgc = (C.c_float * 3)(*[float(x) for x in bg])
        check(self.L.gs_render_fwd(C.byref(self.proj), _ptr(self.sorted_vals), _ptr(self.ranges), self.units.n,
                                   self.W, self.H, bgc, _ptr(self.img), _ptr(self.final_T), _ptr(self.n_contrib),
                                   self.variant, self._sched(), _stream()), "gs_render_fwd")
        return self.img

    def forward(self, params, cams_dev, bg, owned=None):
        self.preprocess(params, cams_dev, owned)
        self.sort()
        return self.render(bg)

    def total_instances(self) -> int:
        """Instances the current projections need (host sum of tiles touched; synchronises)."""
        return int(self.tiles[: self.P].sum(dtype=torch.int64).item()) if self.P else 0

    def fit_capacity(self, params, cams_dev, owned=None, slack: float = 1.25) -> int:
        """Project once and size the instance buffers for these views (outside any graph capture)."""
        self.preprocess(params, cams_dev, owned)
        need = self.total_instances()
        if need > self.cap:
            self.set_capacity(int(need * slack) + 1024)
        return need

    def loss(self, gt: torch.Tensor, mask: torch.Tensor, lam: float):
        check(self.L.gs_loss(_ptr(self.img), _ptr(gt), _ptr(mask), self.units.n, self.W, self.H, float(lam),
                             _ptr(self.loss_ws), self.loss_ws.numel(), _ptr(self.loss_val), _ptr(self.dimg),
                             _stream()), "gs_loss")
        return self.loss_val

    def bg_penalty(self, mask: torch.Tensor, lam: float) -> torch.Tensor:
        """Background-opacity penalty (gs_bg_penalty): adds lam x the mean rendered opacity outside the mask
        to the loss value and returns dpenalty/dT_final, the dT input of the backward calls."""
        if self.dL_dT is None:
            self.dL_dT = torch.zeros((self.units.n, self.H, self.W), dtype=torch.float32, device=self.device)
            self.bg_ws = _alloc_ws(self.L.gs_bg_penalty_workspace_size(self.units.n), self.device)
        check(self.L.gs_bg_penalty(_ptr(self.final_T), _ptr(mask), self.units.n, self.W, self.H, float(lam),
                                   _ptr(self.bg_ws), self.bg_ws.numel(), _ptr(self.loss_val), _ptr(self.dL_dT),
                                   _stream()), "gs_bg_penalty")
        return self.dL_dT

    def blend_backward(self, bg, dimg: torch.Tensor | None = None, dT: torch.Tensor | None = None):
        bgc = (C.c_float * 3)(*[float(x) for x in bg])
        d = self.dimg if dimg is None else dimg
        check(self.L.gs_blend_bwd(C.byref(self.proj), _ptr(self.sorted_vals), _ptr(self.ranges), self.units.n,
                                  self.W, self.H, bgc, _ptr(self.img), _ptr(self.final_T), _ptr(self.n_contrib),
                                  _ptr(d), _ptr(dT), C.byref(self.g2d), self.P, self.variant, self._sched(),
                                  _stream()),
              "gs_blend_bwd")

    def project_backward(self, params, cams_dev):
        check(self.L.gs_project_bwd(_ptr(params), self.N, self.deg, C.byref(self.units.struct), _ptr(cams_dev),
                                    C.byref(self.proj), C.byref(self.g2d), _ptr(self.grads), _stream()),
              "gs_project_bwd")
        return self.grads

    def backward(self, params, cams_dev, bg, dimg: torch.Tensor | None = None, dT: torch.Tensor | None = None):
        bgc = (C.c_float * 3)(*[float(x) for x in bg])
        d = self.dimg if dimg is None else dimg
        check(self.L.gs_render_bwd(_ptr(params), self.N, self.deg, C.byref(self.units.struct), _ptr(cams_dev),
                                   C.byref(self.proj), _ptr(self.sorted_vals), _ptr(self.ranges), self.W, self.H,
                                   bgc, _ptr(self.img), _ptr(self.final_T), _ptr(self.n_contrib), _ptr(d),
                                   _ptr(dT), C.byref(self.g2d), _ptr(self.grads), self.variant, self._sched(),
                                   _stream()),
              "gs_render_bwd")
        return self.grads

    def merge_render(self, params, cam_dev, bg, owned: Owned):
        """Ghost-filtered render of all partitions' splats (one unit over all N Gaussians)."""
        assert self.units.n == 1 and self.P == self.N
        bgc = (C.c_float * 3)(*[float(x) for x in bg])
        check(self.L.gs_merge_render(_ptr(params), self.N, self.deg, C.byref(owned.struct), _ptr(cam_dev), self.W,
                                     self.H, bgc, C.byref(self.proj), self.cap, _ptr(self.sort_ws),
                                     self.sort_ws.numel(), _ptr(self.sorted_vals), _ptr(self.ranges),
                                     _ptr(self.num_instances), _ptr(self.img), _ptr(self.final_T),
                                     _ptr(self.n_contrib), self._sched(), _ptr(self.status), _stream()),
              "gs_merge_render")
        return self.img

    def read_status(self, clear=True) -> int:
        return int(self.L.gs_status_read(_ptr(self.status), 1 if clear else 0, _stream()))

    def blend_pairs(self) -> dict:
        """Work counters of the last forward (diagnostic; synchronises): blended (pixel, record) pairs,
        (pixel, entry) pairs a sequential walk evaluates until each pixel stops, the sum of n_contrib, and
        the two pair counts restricted to entries whose block mask reaches the pixel's 4x4 block."""
        cnt = torch.zeros(5, dtype=torch.int64, device=self.device)
        masks = self.block_masks if self.use_masks else None
        check(self.L.gs_blend_pairs(C.byref(self.proj), _ptr(self.sorted_vals), _ptr(self.ranges), self.units.n,
                                    self.W, self.H, _ptr(self.n_contrib), _ptr(masks), _ptr(cnt), _stream()),
              "gs_blend_pairs")
        c = cnt.tolist()
        return {"blended": int(c[0]), "fwd_pairs": int(c[1]), "bwd_pairs": int(c[2]), "fwd_pairs_masked": int(c[3]),
                "bwd_pairs_masked": int(c[4])}

    def xy64(self) -> np.ndarray:
        """Pixel-space means [P, 2] as float64: the exact sums of the float pairs (synchronises)."""
        a = self.xy.cpu().numpy().astype(np.float64)
        return a[:, :2] + a[:, 2:]

    def instances(self) -> int:
        return int(self.num_instances.item())

    def sorted_lists(self):
        """(sorted record ids [I], ranges [U*n_tiles, 2]) as numpy."""
        I = self.instances()
        return self.sorted_vals[:I].cpu().numpy().astype(np.int64), self.ranges.cpu().numpy().astype(np.int64)


class RasterizeFunction(torch.autograd.Function):
    """img = rasterize(params); backward through gs_render_bwd.

    ``frame`` holds the buffers; the returned image is a copy so the frame can
    be reused.  Gradients flow to ``params`` only (cameras are fixed)."""

    @staticmethod
    def forward(ctx, params, frame: Frame, cams_dev, bg):
        frame.forward(params.detach().contiguous(), cams_dev, bg)
        ctx.frame, ctx.cams, ctx.bg = frame, cams_dev, bg
        ctx.save_for_backward(params)
        return frame.img.clone()

    @staticmethod
    def backward(ctx, dimg):
        (params,) = ctx.saved_tensors
        g = ctx.frame.backward(params.detach().contiguous(), ctx.cams, ctx.bg, dimg.contiguous())
        return g.clone(), None, None, None


def rasterize(params, frame: Frame, cams_dev, bg):
    return RasterizeFunction.apply(params, frame, cams_dev, bg)


# ---------------------------------------------------------------- optimiser
@dataclass
class LearningRates:
    """Per-group Adam learning rates (3D-GS defaults; the paper states none).

    means decay log-linearly from mean_init * extent to mean_final * extent."""

    mean_init: float = 1.6e-4
    mean_final: float = 1.6e-6
    scale: float = 5e-3
    opacity: float = 5e-2
    rotation: float = 1e-3
    sh_dc: float = 2.5e-3
    sh_rest: float = 2.5e-3 / 20.0

    def tables(self, sh_degree: int, extent: float = 1.0):
        npl = param_planes(sh_degree)
        init = np.zeros((npl, 4), np.float32)
        fin = np.zeros((npl, 4), np.float32)
        init[0, :3] = self.mean_init * extent
        fin[0, :3] = self.mean_final * extent
        init[1, :3] = self.scale
        init[1, 3] = self.opacity
        init[2, :] = self.rotation
        sh = np.full((npl - 3) * 4, self.sh_rest, np.float32)
        sh[:3] = self.sh_dc
        init[3:] = sh.reshape(npl - 3, 4)
        fin[1:] = init[1:]
        return init, fin


class Adam:
    """Adam state (m, v, step counter on the device) for a planes tensor."""

    def __init__(self, params: torch.Tensor, sh_degree: int, lrs: LearningRates | None = None, extent: float = 1.0,
                 lr_steps: int = 30000, betas=(0.9, 0.999), eps: float = 1e-15):
        self.L = _lib.load()
        self.params = params
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.step_dev = torch.zeros(1, dtype=torch.int32, device=params.device)
        # device status word of step(): GS_ERR_NONFINITE when a gradient value was not finite
        self.status = torch.zeros(1, dtype=torch.int32, device=params.device)
        # fused_step: Gaussians without gradient in a step keep their state (sparse Adam)
        self.sparse = False
        init, fin = (lrs or LearningRates()).tables(sh_degree, extent)
        self.lr_init = np.ascontiguousarray(init.reshape(-1))
        self.lr_final = np.ascontiguousarray(fin.reshape(-1))
        self.lr_steps = int(lr_steps)
        self.b1, self.b2 = betas
        self.eps = eps

    def fused_step(self, frame: "Frame", cams_dev, keep_grads: bool = False, next_cams_dev=None):
        """Projection backward of ``frame``'s screen-space gradients fused with this Adam step
        (gs_project_bwd_adam); ``frame.grads`` receives the gradient only if keep_grads.  With next_cams_dev
        the same kernel also projects the updated Gaussians for those cameras into ``frame``'s records
        (gs_project_bwd_adam_next), so the next step needs no preprocess call."""
        n = self.params.shape[1]
        common = (_ptr(self.params), n, frame.deg, C.byref(frame.units.struct), _ptr(cams_dev), C.byref(frame.proj),
                  C.byref(frame.g2d), _ptr(self.m), _ptr(self.v), self.lr_init.ctypes.data_as(_lib.c_f32p),
                  self.lr_final.ctypes.data_as(_lib.c_f32p), self.lr_steps, self.b1, self.b2, self.eps,
                  _ptr(self.step_dev), _ptr(frame.grads) if keep_grads else None, int(self.sparse))
        if next_cams_dev is None:
            check(self.L.gs_project_bwd_adam(*common, _ptr(frame.status), _stream()), "gs_project_bwd_adam")
        else:
            check(self.L.gs_project_bwd_adam_next(*common, _ptr(next_cams_dev), frame.W, frame.H, _ptr(frame.status),
                                                  _stream()), "gs_project_bwd_adam_next")
        check(self.L.gs_step_advance(_ptr(self.step_dev), _stream()), "gs_step_advance")

    def state_dict(self) -> dict:
        """Optimiser state for a checkpoint: moments and the device step counter (copies)."""
        return {"m": self.m.clone(), "v": self.v.clone(), "step": self.step_dev.clone()}

    def load_state_dict(self, st: dict):
        self.m.copy_(st["m"])
        self.v.copy_(st["v"])
        self.step_dev.copy_(st["step"])

    def step(self, grads: torch.Tensor, zero_grad: bool = False):
        npl, n = self.params.shape[0], self.params.shape[1]
        check(self.L.gs_adam_step(_ptr(self.params), _ptr(grads), _ptr(self.m), _ptr(self.v), n, npl,
                                  self.lr_init.ctypes.data_as(_lib.c_f32p), self.lr_final.ctypes.data_as(_lib.c_f32p),
                                  self.lr_steps, self.b1, self.b2, self.eps, _ptr(self.step_dev), int(zero_grad),
                                  _ptr(self.status), _stream()), "gs_adam_step")
        check(self.L.gs_step_advance(_ptr(self.step_dev), _stream()), "gs_step_advance")
