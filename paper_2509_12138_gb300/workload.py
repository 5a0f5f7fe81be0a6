"""Synthetic isosurface training workloads on the device.

The paper's datasets (isosurfaces of 4M-107M points, Sec. III) are not
available; a Richtmyer-Meshkov-like perturbed interface (synth.interface_points)
stands in.  Ground-truth images are renders of a surfel set on the same points
(flat, opaque, normal-aligned Gaussians with the points' Lambert colours),
made with this library's own forward pass; the background mask of a view is
the GT coverage, 1 - T_final >= 1/255 (Sec. II, "Image Rendering and Masking").
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

import synth

from .raster import Frame, Units, pack_cameras, pack_params

Y00 = 0.28209479177387814


def spacing_estimate(normals: np.ndarray, n: int) -> float:
    """Mean 3-NN distance of n uniform samples on the unit-square height field:
    area = mean(1/n_z); for a planar Poisson process of density lam the mean of the
    first three NN distances is (0.5 + 0.75 + 0.9375) / 3 / sqrt(lam)."""
    area = float(np.mean(1.0 / np.abs(np.asarray(normals, np.float64)[:, 2])))
    lam = n / area
    return (0.5 + 0.75 + 0.9375) / 3.0 / math.sqrt(lam)


def gaussians_from_points(pts, colors, log_scales, quats, logit, sh_degree: int):
    n = pts.shape[0]
    sh = np.zeros((n, (sh_degree + 1) ** 2, 3), np.float32)
    sh[:, 0, :] = (colors - 0.5) / Y00
    return dict(means=pts.astype(np.float32), log_scales=np.asarray(log_scales, np.float32),
                quats=np.asarray(quats, np.float32), logit_opacity=np.asarray(logit, np.float32), sh=sh)


def gt_surfels(pts, nrm, colors, spacing: float, sh_degree: int = 0):
    n = pts.shape[0]
    ls = np.tile(np.log([spacing, spacing, 0.1 * spacing]).astype(np.float32), (n, 1))
    q = synth.surfel_quats(nrm)
    logit = np.full(n, math.log(0.99 / 0.01), np.float32)
    return gaussians_from_points(pts, colors, ls, q, logit, sh_degree)


def plain_init(pts, colors, log_scale, sh_degree: int = 3, opacity: float = 0.1):
    """Plain isosurface initialisation: isotropic scale, identity rotation, opacity 0.1, DC colour."""
    n = pts.shape[0]
    ls = np.broadcast_to(np.asarray(log_scale, np.float32).reshape(-1, 1), (n, 3)).copy() \
        if np.ndim(log_scale) else np.full((n, 3), float(log_scale), np.float32)
    q = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1))
    logit = np.full(n, math.log(opacity / (1 - opacity)), np.float32)
    return gaussians_from_points(pts, colors, ls, q, logit, sh_degree)


@dataclass
class Scene:
    n: int
    sh_degree: int
    width: int
    height: int
    cams: synth.Cameras
    cams_dev: torch.Tensor      # [V * 96] bytes of gs_camera
    gt: torch.Tensor            # [V, 3, H, W]
    mask: torch.Tensor          # [V, H, W] uint8
    init: dict                  # numpy Gaussian dict (plain init)
    pts: np.ndarray
    nrm: np.ndarray
    colors: np.ndarray
    spacing: float
    bg: tuple = (1.0, 1.0, 1.0)

    def cam(self, v: int) -> torch.Tensor:
        return self.cams_dev[v * 96:(v + 1) * 96]


def render_gt(gauss: dict, cams: synth.Cameras, sh_degree: int, bg, device="cuda", max_instances=None):
    """GT images and masks of every camera, rendered one view at a time."""
    n = gauss["means"].shape[0]
    W, H = cams.width, cams.height
    fr = Frame(n, Units.single(n), W, H, sh_degree, device=device, with_backward=False, with_loss=False,
               max_instances=max_instances)
    params = pack_params(gauss, sh_degree, device)
    camd = pack_cameras(cams, device)
    V = len(cams)
    gt = torch.empty((V, 3, H, W), dtype=torch.float32, device=device)
    mask = torch.empty((V, H, W), dtype=torch.uint8, device=device)
    for v in range(V):
        fr.forward(params, camd[v * 96:(v + 1) * 96], bg)
        gt[v] = fr.img[0]
        mask[v] = (1.0 - fr.final_T[0]) >= (1.0 / 255.0)
    st = fr.read_status()
    if st != 0:
        raise RuntimeError(f"GT render status {st}")
    del fr, params
    return gt, mask


@dataclass
class PointScene:
    """The host side of an isosurface scene: points, cameras and the plain initialisation, no GT images
    (for consumers that render what they need themselves, such as the oracle's timed sample)."""
    n: int
    sh_degree: int
    width: int
    height: int
    cams: synth.Cameras
    init: dict
    pts: np.ndarray
    nrm: np.ndarray
    colors: np.ndarray
    spacing: float


def isosurface_points(n: int, n_modes: int, n_views: int, width: int, height: int, sh_degree: int = 3,
                      seed: int = 0, radius: float = 1.5, init_log_scale=None, spatial: bool = True) -> PointScene:
    """spatial: store the points in Z-order (synth.spatial_order), the cell-by-cell order in which an
    isosurface extraction emits them; False keeps the sampler's random order."""
    pts, nrm, _ = synth.interface_points(n, n_modes, seed)
    if spatial:
        o = synth.spatial_order(pts)
        pts, nrm = pts[o], nrm[o]
    colors = synth.lambert_colors(pts, nrm)
    spacing = spacing_estimate(nrm, n)
    cams = synth.orbital_cameras(n_views, radius, center=(0.5, 0.5, 0.5), width=width, height=height)
    ls = math.log(spacing) if init_log_scale is None else init_log_scale
    init = plain_init(pts, colors, ls, sh_degree)
    return PointScene(n=n, sh_degree=sh_degree, width=width, height=height, cams=cams, init=init, pts=pts, nrm=nrm,
                      colors=colors, spacing=spacing)


def isosurface_scene(n: int, n_modes: int, n_views: int, width: int, height: int, sh_degree: int = 3,
                     seed: int = 0, radius: float = 1.5, device="cuda", init_log_scale=None,
                     spatial: bool = True) -> Scene:
    """The points of isosurface_points with every view's GT image and mask rendered on the device."""
    ps = isosurface_points(n, n_modes, n_views, width, height, sh_degree, seed, radius, init_log_scale, spatial)
    gt, mask = render_gt(gt_surfels(ps.pts, ps.nrm, ps.colors, ps.spacing), ps.cams, 0, (1.0, 1.0, 1.0), device,
                         max_instances=max(8 * n, 1 << 20))
    return Scene(n=n, sh_degree=sh_degree, width=width, height=height, cams=ps.cams,
                 cams_dev=pack_cameras(ps.cams, device), gt=gt, mask=mask, init=ps.init, pts=ps.pts, nrm=ps.nrm,
                 colors=ps.colors, spacing=ps.spacing)


@dataclass
class PartitionedScene:
    part: object                 # partition.Partition
    sh_degree: int
    width: int
    height: int
    cams: synth.Cameras
    cams_dev: torch.Tensor
    gt: torch.Tensor             # [n_parts, V, 3, H, W]: each partition's own GT (owned + ghost points)
    mask: torch.Tensor           # [n_parts, V, H, W]
    gt_full: torch.Tensor        # [V, 3, H, W]: GT of the whole scene (for the merged render)
    mask_full: torch.Tensor
    init: dict                   # plain init, partition-major
    pts: np.ndarray
    spacing: float
    bg: tuple = (1.0, 1.0, 1.0)
    nrm: np.ndarray | None = None  # surface normals of pts

    @property
    def offsets(self):
        return self.part.offsets


def partitioned_scene(slab_counts, n_modes: int, n_views: int, width: int, height: int, n_parts: int = 8,
                      ghost: float = 0.05, sh_degree: int = 3, seed: int = 0, radius: float = 1.5,
                      device="cuda", init_scale: float = 1.0) -> PartitionedScene:
    """The interface split into x-slabs with ghost layers; uneven slab populations from a piecewise
    constant x-density (slab_counts points per slab).  init_scale: factor on the plain initialisation's
    isotropic scale (the mean 3-NN spacing)."""
    from .partition import slab_partition
    pts, nrm, _ = synth.slab_density_points(n_modes=n_modes, slab_counts=slab_counts, seed=seed)
    o = synth.spatial_order(pts)  # Z-order, as an isosurface extraction emits the points
    pts, nrm = pts[o], nrm[o]
    n = pts.shape[0]
    colors = synth.lambert_colors(pts, nrm)
    spacing = spacing_estimate(nrm, n)
    cams = synth.orbital_cameras(n_views, radius, center=(0.5, 0.5, 0.5), width=width, height=height)
    part = slab_partition(pts, n_parts, ghost)
    H, W = height, width
    gt = torch.empty((n_parts, n_views, 3, H, W), dtype=torch.float32, device=device)
    mask = torch.empty((n_parts, n_views, H, W), dtype=torch.uint8, device=device)
    for k in range(n_parts):
        idx = part.members[k]
        g, m = render_gt(gt_surfels(pts[idx], nrm[idx], colors[idx], spacing), cams, 0, (1.0, 1.0, 1.0), device,
                         max_instances=max(8 * len(idx), 1 << 20))
        gt[k], mask[k] = g, m
    gt_full, mask_full = render_gt(gt_surfels(pts, nrm, colors, spacing), cams, 0, (1.0, 1.0, 1.0), device,
                                   max_instances=max(8 * n, 1 << 20))
    order = part.order
    init = plain_init(pts[order], colors[order], math.log(spacing * init_scale), sh_degree)
    return PartitionedScene(part=part, sh_degree=sh_degree, width=W, height=H, cams=cams,
                            cams_dev=pack_cameras(cams, device), gt=gt, mask=mask, gt_full=gt_full,
                            mask_full=mask_full, init=init, pts=pts, spacing=spacing, nrm=nrm)


def _spread2(v: torch.Tensor) -> torch.Tensor:
    """x in [0, 1) quantised to 16 bits, its bits moved to the even positions 0, 2, ..., 30 (int64)."""
    q = (v.double() * 65535.0).round().long().clamp_(0, 65535)
    q = (q | (q << 8)) & 0x00FF00FF
    q = (q | (q << 4)) & 0x0F0F0F0F
    q = (q | (q << 2)) & 0x33333333
    q = (q | (q << 1)) & 0x55555555
    return q


def interface_gaussians_device(n: int, n_modes: int, seed: int, sh_degree: int = 3, device="cuda",
                               chunk: int = 1 << 24):
    """Plain-initialised Gaussians on the perturbed interface generated directly on the device (for
    render-only scenes too large to stage through host memory).  Same field as synth.interface_points
    (the amplitudes, directions and phases come from synth's seeded streams); positions from a seeded
    torch generator.  Returns (planes [n_planes, n, 4], x coordinates [n])."""
    from .raster import param_planes
    s = synth.streams(seed, ["amp", "dir", "phase"])
    k = torch.arange(1, n_modes + 1, dtype=torch.float64)
    amp = torch.from_numpy(s["amp"].uniform(0.0, 1.0, n_modes)) / k
    theta = torch.from_numpy(s["dir"].uniform(0.0, 2.0 * math.pi, n_modes))
    phase = torch.from_numpy(s["phase"].uniform(0.0, 2.0 * math.pi, n_modes))
    kx, ky = (k * torch.cos(theta)).float().to(device), (k * torch.sin(theta)).float().to(device)
    amp, phase = amp.float().to(device), phase.float().to(device)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    npl = param_planes(sh_degree)
    params = torch.zeros((npl, n, 4), dtype=torch.float32, device=device)
    xs = torch.empty(n, dtype=torch.float32, device=device)
    ys = torch.empty(n, dtype=torch.float32, device=device)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        xs[a:b] = torch.rand(b - a, generator=gen, device=device)
        ys[a:b] = torch.rand(b - a, generator=gen, device=device)
    # Z-order over (x, y) (the interface is a height field): the cell-by-cell order of an extraction
    o = torch.argsort(_spread2(xs) | (_spread2(ys) << 1), stable=True)
    xs, ys = xs[o], ys[o]
    del o
    area = 0.0
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        x, y = xs[a:b], ys[a:b]
        arg = 2.0 * math.pi * (x[:, None] * kx + y[:, None] * ky) + phase
        h = 0.1 * (torch.sin(arg) * amp).sum(1)
        dh = 0.1 * torch.cos(arg) * amp * 2.0 * math.pi
        hx, hy = (dh * kx).sum(1), (dh * ky).sum(1)
        nz = 1.0 / torch.sqrt(hx * hx + hy * hy + 1.0)
        area += float((1.0 / nz).sum())
        z = 0.5 + h
        params[0, a:b, 0], params[0, a:b, 1], params[0, a:b, 2] = x, y, z
        zn = (z - 0.2) / 0.6
        ndl = torch.abs((-hx * 0.3 - hy * 0.5 + 0.8) * nz / math.sqrt(0.98))
        shade = 0.2 + 0.8 * ndl
        col = torch.stack([0.2 + 0.75 * zn, 0.4 + 0.2 * zn, 0.9 - 0.7 * zn], 1) * shade[:, None]
        dc = (col.clamp(0, 1) - 0.5) / Y00
        params[3, a:b, 0:3] = dc
    spacing = (0.5 + 0.75 + 0.9375) / 3.0 / math.sqrt(n / (area / n))
    params[1, :, 0:3] = math.log(spacing)
    params[1, :, 3] = math.log(0.5 / 0.5)  # opacity 0.5 for a visible render-only scene
    params[2, :, 0] = 1.0
    return params, xs


def partition_device(params: torch.Tensor, xs: torch.Tensor, n_parts: int = 8, ghost: float = 0.05):
    """Partition-major copy of a planes tensor by x-slabs with ghost layers (as partition.slab_partition),
    built on the device.  Returns (planes, part_offsets, owned boxes, closed_hi)."""
    from .partition import BIG
    edges = np.linspace(0.0, 1.0, n_parts + 1)
    w = 1.0 / n_parts
    idx = []
    for k in range(n_parts):
        a = edges[k] - (ghost * w if k > 0 else 0.0)
        b = edges[k + 1] + (ghost * w if k < n_parts - 1 else 0.0)
        sel = (xs >= a) & ((xs <= b) if k == n_parts - 1 else (xs < b))
        idx.append(torch.nonzero(sel).squeeze(1))
    offsets = np.concatenate([[0], np.cumsum([len(i) for i in idx])]).astype(np.int64)
    order = torch.cat(idx)
    out = params[:, order].contiguous()
    boxes = np.zeros((n_parts, 6), np.float32)
    boxes[:, 0], boxes[:, 3] = edges[:-1], edges[1:]
    boxes[:, 1] = boxes[:, 2] = -BIG
    boxes[:, 4] = boxes[:, 5] = BIG
    closed = np.full(n_parts, 0b110, np.int32)
    closed[-1] |= 1
    return out, offsets, boxes, closed
