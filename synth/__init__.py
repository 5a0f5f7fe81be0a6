"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only *makes data*: isosurface point samples, their normals and
Lambert colours, orbital cameras, random Gaussian parameter sets and the
random perturbations used to build training targets.  It holds none of the
rasterizer's arithmetic (projection, binning, blending, loss, gradients,
optimiser); those live in the CUDA library and, independently, in the oracle.

Every generator takes an integer seed and derives one independent
``numpy.random.Generator`` per drawn quantity with ``SeedSequence.spawn``, so
adding a quantity never changes the others.

Workloads (paper Sec. III evaluates isosurfaces of 4M-107M points rendered
from an orbital camera set; the datasets themselves are not available, so the
analytic interfaces below stand in for them):

* ``sphere_points``      -- points uniform on the unit sphere (small workload).
* ``interface_points``   -- a Richtmyer-Meshkov-like perturbed interface:
  the 0.5 isosurface of f(x, y, z) = z - 0.1 * sum_k a_k sin(2 pi (kx x + ky y) + phi_k)
  on the unit square, with a_k ~ U(0, 1) / k, wave vectors of magnitude k in a
  random direction and random phases.  Points are sampled with (x, y) ~ U(0,1)^2
  and z exact, so they lie exactly on the isosurface; normals are analytic.
* ``orbital_cameras``    -- the "structured orbital set of synthetic camera
  views" of Sec. II, realised as a golden-angle (Fibonacci) sphere of viewpoints
  looking at the scene centre.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "streams",
    "orbital_cameras",
    "sphere_points",
    "interface_points",
    "lambert_colors",
    "random_gaussians",
    "target_perturbation",
    "slab_density_points",
    "surfel_quats",
    "Cameras",
]


def streams(seed: int, names):
    """One independent Generator per name, derived from ``seed`` by SeedSequence.spawn."""
    names = list(names)
    children = np.random.SeedSequence(seed).spawn(len(names))
    return {n: np.random.default_rng(c) for n, c in zip(names, children)}


@dataclass
class Cameras:
    """A batch of pinhole cameras (float32, world -> camera).

    viewmat[i] is the 3x4 row-major [R | t]; camera space has +x right, +y down
    and +z forward, so a world point X maps to pixel
    (fx * x / z + cx, fy * y / z + cy) with X_cam = R X + t.
    """

    viewmat: np.ndarray  # [n, 3, 4]
    fx: np.ndarray  # [n]
    fy: np.ndarray
    cx: np.ndarray
    cy: np.ndarray
    tan_fovx: np.ndarray
    tan_fovy: np.ndarray
    campos: np.ndarray  # [n, 3]
    znear: float
    width: int
    height: int

    def __len__(self):
        return self.viewmat.shape[0]

    def subset(self, idx):
        idx = np.atleast_1d(np.asarray(idx))
        return Cameras(self.viewmat[idx], self.fx[idx], self.fy[idx], self.cx[idx], self.cy[idx],
                       self.tan_fovx[idx], self.tan_fovy[idx], self.campos[idx], self.znear,
                       self.width, self.height)

    @staticmethod
    def concat(cams):
        cams = list(cams)
        w, h = cams[0].width, cams[0].height
        assert all(c.width == w and c.height == h for c in cams)
        cat = lambda f: np.concatenate([getattr(c, f) for c in cams], axis=0)
        return Cameras(cat("viewmat"), cat("fx"), cat("fy"), cat("cx"), cat("cy"), cat("tan_fovx"),
                       cat("tan_fovy"), cat("campos"), cams[0].znear, w, h)


def _look_at(eye, target):
    f = target - eye
    f = f / np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0])
    if abs(float(f @ up)) > 0.99:
        up = np.array([0.0, 1.0, 0.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)  # image "down"; (r, d, f) is right-handed
    R = np.stack([r, d, f], axis=0)
    t = -R @ eye
    return R, t


def orbital_cameras(n: int, radius: float, center=(0.0, 0.0, 0.0), width: int = 128,
                    height: int = 128, fovy_deg: float = 60.0, znear: float = 0.2) -> Cameras:
    """``n`` viewpoints on a golden-angle sphere of ``radius`` about ``center``.

    Vertical field of view ``fovy_deg``; fx = fy = height / (2 tan(fovy / 2));
    principal point ((W - 1) / 2, (H - 1) / 2) so that pixel (px, py) sits at
    integer coordinates.
    """
    center = np.asarray(center, dtype=np.float64)
    golden = math.pi * (3.0 - math.sqrt(5.0))
    vm = np.zeros((n, 3, 4))
    campos = np.zeros((n, 3))
    for k in range(n):
        z = 1.0 - (2.0 * k + 1.0) / n
        rr = math.sqrt(max(0.0, 1.0 - z * z))
        phi = golden * k
        eye = center + radius * np.array([rr * math.cos(phi), rr * math.sin(phi), z])
        R, t = _look_at(eye, center)
        vm[k, :, :3] = R
        vm[k, :, 3] = t
        campos[k] = eye
    tan_y = math.tan(math.radians(fovy_deg) / 2.0)
    f = height / (2.0 * tan_y)
    tan_x = (width / 2.0) / f
    ones = np.ones(n)
    return Cameras(
        viewmat=vm.astype(np.float32),
        fx=(f * ones).astype(np.float32),
        fy=(f * ones).astype(np.float32),
        cx=((width - 1) / 2.0 * ones).astype(np.float32),
        cy=((height - 1) / 2.0 * ones).astype(np.float32),
        tan_fovx=(tan_x * ones).astype(np.float32),
        tan_fovy=(tan_y * ones).astype(np.float32),
        campos=campos.astype(np.float32),
        znear=float(znear),
        width=int(width),
        height=int(height),
    )


def sphere_points(n: int, seed: int = 0):
    """Points uniform on the unit sphere (normalised N(0, I) samples) and their normals."""
    g = streams(seed, ["points"])["points"]
    p = g.standard_normal((n, 3))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    return p.astype(np.float32), p.astype(np.float32)


def interface_points(n: int, n_modes: int, seed: int = 0, x_density=None):
    """Samples of the perturbed-interface isosurface and analytic unit normals.

    ``x_density`` optionally gives a piecewise-constant density over equal-width
    x bins (used to make uneven slab partitions); otherwise x ~ U(0, 1).
    Returns (points [n,3] f32, normals [n,3] f32, field dict).
    """
    s = streams(seed, ["amp", "dir", "phase", "x", "y"])
    k = np.arange(1, n_modes + 1, dtype=np.float64)
    amp = s["amp"].uniform(0.0, 1.0, n_modes) / k
    theta = s["dir"].uniform(0.0, 2.0 * math.pi, n_modes)
    phase = s["phase"].uniform(0.0, 2.0 * math.pi, n_modes)
    kx, ky = k * np.cos(theta), k * np.sin(theta)
    if x_density is None:
        x = s["x"].uniform(0.0, 1.0, n)
    else:
        w = np.asarray(x_density, dtype=np.float64)
        w = w / w.sum()
        nb = len(w)
        counts = np.floor(w * n).astype(np.int64)
        counts[: n - counts.sum()] += 1
        bins = np.repeat(np.arange(nb), counts)
        x = (bins + s["x"].uniform(0.0, 1.0, n)) / nb
    y = s["y"].uniform(0.0, 1.0, n)
    h = np.empty(n)
    hx = np.empty(n)
    hy = np.empty(n)
    for a in range(0, n, 1 << 20):  # chunks keep the n x modes temporaries small
        b = min(n, a + (1 << 20))
        arg = 2.0 * math.pi * (np.outer(x[a:b], kx) + np.outer(y[a:b], ky)) + phase
        h[a:b] = 0.1 * (np.sin(arg) * amp).sum(axis=1)
        dh = 0.1 * np.cos(arg) * amp * 2.0 * math.pi
        hx[a:b] = (dh * kx).sum(axis=1)
        hy[a:b] = (dh * ky).sum(axis=1)
    z = 0.5 + h
    pts = np.stack([x, y, z], axis=1)
    nrm = np.stack([-hx, -hy, np.ones_like(hx)], axis=1)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    field = dict(amp=amp, kx=kx, ky=ky, phase=phase)
    return pts.astype(np.float32), nrm.astype(np.float32), field


def slab_density_points(n_modes: int, slab_counts, seed: int = 0):
    """Interface samples whose x-distribution gives the requested per-slab counts.

    ``slab_counts`` are the wanted counts for equal-width x-slabs of [0, 1]
    (their sum is the total); the density is piecewise constant per slab.
    """
    slab_counts = np.asarray(slab_counts, dtype=np.float64)
    return interface_points(int(slab_counts.sum()), n_modes, seed, x_density=slab_counts)


def _spread3(v):
    """Bits 0..9 of v moved to bits 0, 3, 6, ..., 27 (uint64)."""
    v = v & np.uint64(0x3FF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x030000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x0300F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x030C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x09249249)
    return v


def spatial_order(points):
    """Permutation that puts points in Z-order (Morton order of a 1024^3 grid over their bounding
    box), the cell-by-cell coherence of the points an isosurface extraction emits.  Stable."""
    p = np.asarray(points, dtype=np.float64)
    if p.shape[0] == 0:
        return np.zeros(0, dtype=np.int64)
    lo, hi = p.min(axis=0), p.max(axis=0)
    q = ((p - lo) / np.maximum(hi - lo, 1e-30) * 1023.0).round().astype(np.uint64)
    code = _spread3(q[:, 0]) | (_spread3(q[:, 1]) << np.uint64(1)) | (_spread3(q[:, 2]) << np.uint64(2))
    return np.argsort(code, kind="stable")


def lambert_colors(points, normals):
    """Albedo ramp over normalised height, shaded by a fixed directional light.

    albedo = lerp((0.2, 0.4, 0.9), (0.95, 0.6, 0.2), z_norm);
    colour = albedo * (0.2 + 0.8 * max(0, n . L)), L = normalise(0.3, 0.5, 0.8).
    Two-sided: the normal is flipped toward the light.
    """
    p = np.asarray(points, dtype=np.float64)
    nrm = np.asarray(normals, dtype=np.float64)
    z = p[:, 2]
    zn = (z - z.min()) / max(1e-12, float(z.max() - z.min()))
    lo = np.array([0.2, 0.4, 0.9])
    hi = np.array([0.95, 0.6, 0.2])
    albedo = lo[None] + (hi - lo)[None] * zn[:, None]
    L = np.array([0.3, 0.5, 0.8])
    L /= np.linalg.norm(L)
    ndl = np.abs(nrm @ L)
    col = albedo * (0.2 + 0.8 * ndl)[:, None]
    return col.astype(np.float32)


def surfel_quats(normals):
    """Unit quaternions (w, x, y, z) rotating +z onto each normal (GT surfel orientation)."""
    n = np.asarray(normals, np.float64)
    q = np.stack([1.0 + n[:, 2], -n[:, 1], n[:, 0], np.zeros(len(n))], axis=1)
    bad = q[:, 0] < 1e-9  # normal = -z: rotate by pi about x
    q[bad] = [0.0, 1.0, 0.0, 0.0]
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def random_gaussians(n: int, sh_degree: int = 3, seed: int = 0, center=(0.0, 0.0, 0.0),
                     extent: float = 1.0, log_scale_range=(-4.0, -2.0), sh_scale: float = 0.3):
    """Random, well-conditioned Gaussian parameter sets for parity / gradient tests.

    Returns dict of float32 arrays: means [n,3], log_scales [n,3], quats [n,4]
    (w, x, y, z, not normalised), logit_opacity [n], sh [n, (d+1)^2, 3].
    """
    s = streams(seed, ["mean", "scale", "quat", "opacity", "sh"])
    c = np.asarray(center, dtype=np.float64)
    means = c + s["mean"].uniform(-extent, extent, (n, 3))
    log_scales = s["scale"].uniform(log_scale_range[0], log_scale_range[1], (n, 3))
    quats = s["quat"].standard_normal((n, 4))
    quats *= s["quat"].uniform(0.5, 2.0, (n, 1)) / np.linalg.norm(quats, axis=1, keepdims=True)
    logit = s["opacity"].uniform(-2.0, 3.0, n)
    nc = (sh_degree + 1) ** 2
    sh = s["sh"].standard_normal((n, nc, 3)) * sh_scale
    sh[:, 0, :] = s["sh"].uniform(-1.0, 1.0, (n, 3))
    return dict(
        means=means.astype(np.float32),
        log_scales=log_scales.astype(np.float32),
        quats=quats.astype(np.float32),
        logit_opacity=logit.astype(np.float32),
        sh=sh.astype(np.float32),
    )


def target_perturbation(n: int, seed: int = 0):
    """Random draws that turn a Gaussian set into a training target (small workload).

    mean noise ~ N(0, 0.01^2), log-scale noise ~ N(0, 0.1^2), target RGB ~ U(0.1, 0.9).
    """
    s = streams(seed, ["mean", "scale", "rgb"])
    return dict(
        mean_noise=(0.01 * s["mean"].standard_normal((n, 3))).astype(np.float32),
        log_scale_noise=(0.1 * s["scale"].standard_normal((n, 3))).astype(np.float32),
        rgb=s["rgb"].uniform(0.1, 0.9, (n, 3)).astype(np.float32),
    )
