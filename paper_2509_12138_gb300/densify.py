"""Adaptive density control of 3D Gaussian Splatting over libgs.

Every training step adds its view's statistics (gs_densify_stats); every ``interval`` steps within
[``start``, ``stop``) the Gaussians are cloned, split and pruned (gs_densify_plan / gs_densify_apply)
into newly allocated parameter and Adam planes; every ``reset_interval`` steps the opacities are reset
(gs_opacity_reset).  The rules are those of 3D-GS as stated in include/gs.h; the split draws come from a
seeded torch generator on the device.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import GsDensifyCfg, check
from .raster import _ptr, _stream


@dataclass
class DensifyConfig:
    grad_threshold: float = 2e-4
    percent_dense: float = 0.01
    min_opacity: float = 0.005
    max_screen: float = 20.0
    extent: float = 1.0
    start: int = 500
    stop: int = 15000
    interval: int = 100
    reset_interval: int = 3000
    reset_opacity: float = 0.01


class Densifier:
    def __init__(self, n_gauss: int, cfg: DensifyConfig | None = None, device="cuda", seed: int = 0):
        self.L = _lib.load()
        self.cfg = cfg or DensifyConfig()
        self.device = torch.device(device)
        self.gen = torch.Generator(device=self.device)
        self.gen.manual_seed(seed)
        self.counts = torch.zeros(3, dtype=torch.int32, device=self.device)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self._alloc(n_gauss)

    def _alloc(self, n: int):
        self.n = int(n)
        f = dict(dtype=torch.float32, device=self.device)
        self.grad_accum = torch.zeros(max(self.n, 1), **f)
        self.denom = torch.zeros(max(self.n, 1), **f)
        self.max_radius = torch.zeros(max(self.n, 1), **f)

    def accumulate(self, frame):
        """Add the statistics of the frame's last backward (its units' screen-space gradients)."""
        check(self.L.gs_densify_stats(C.byref(frame.proj), C.byref(frame.g2d), C.byref(frame.units.struct), frame.W,
                                      frame.H, _ptr(self.grad_accum), _ptr(self.denom), _ptr(self.max_radius),
                                      _stream()), "gs_densify_stats")

    def due(self, step: int) -> bool:
        c = self.cfg
        return c.start <= step < c.stop and step % c.interval == 0

    def reset_due(self, step: int) -> bool:
        c = self.cfg
        return step > 0 and step < c.stop and step % c.reset_interval == 0

    def plan(self, params: torch.Tensor, step: int):
        """(kept, cloned, split) for the current statistics (synchronises)."""
        c = self.cfg
        cfg = GsDensifyCfg(c.grad_threshold, c.percent_dense, c.min_opacity, c.max_screen, c.extent, int(step),
                           c.reset_interval)
        n = params.shape[1]
        assert n == self.n
        ws = self.L.gs_densify_workspace_size(n)
        self.ws = torch.empty(ws + 256, dtype=torch.uint8, device=self.device)
        off = (-self.ws.data_ptr()) % 256
        self.ws_ptr, self.ws_bytes = self.ws.data_ptr() + off, ws
        check(self.L.gs_densify_plan(_ptr(params), n, _ptr(self.grad_accum), _ptr(self.denom), _ptr(self.max_radius),
                                     C.byref(cfg), C.c_void_p(self.ws_ptr), self.ws_bytes, _ptr(self.counts),
                                     _stream()), "gs_densify_plan")
        kept, cloned, split = (int(x) for x in self.counts.tolist())
        return kept, cloned, split

    def apply(self, params: torch.Tensor, m: torch.Tensor, v: torch.Tensor, deg: int, counts, z=None):
        """New (params, m, v) planes for the last plan; z: [n, 2, 3] standard normal draws (drawn here if None)."""
        kept, cloned, split = counts
        n = params.shape[1]
        n_out = kept + cloned + 2 * split
        if z is None:
            z = torch.randn((n, 2, 3), generator=self.gen, device=self.device, dtype=torch.float32)
        shape = (params.shape[0], max(n_out, 1), 4)
        out = [torch.empty(shape, dtype=torch.float32, device=self.device) for _ in range(3)]
        check(self.L.gs_densify_apply(_ptr(params), _ptr(m), _ptr(v), n, deg, _ptr(z), C.c_void_p(self.ws_ptr),
                                      self.ws_bytes, _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), n_out,
                                      _ptr(self.status), _stream()), "gs_densify_apply")
        self._alloc(n_out)  # statistics restart from zero for the new set
        return tuple(o[:, :n_out].contiguous() if n_out == 0 else o for o in out)

    def reset_opacity(self, params: torch.Tensor, m: torch.Tensor, v: torch.Tensor):
        check(self.L.gs_opacity_reset(_ptr(params), _ptr(m), _ptr(v), params.shape[1], self.cfg.reset_opacity,
                                      _stream()), "gs_opacity_reset")
