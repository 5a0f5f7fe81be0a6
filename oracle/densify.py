"""Adaptive density control of 3D Gaussian Splatting, plain numpy -- TEST INFRASTRUCTURE ONLY.

The paper trains each partition with standard 3D-GS (Sec. II, "Parallel Training"), whose optimisation
periodically clones, splits and prunes Gaussians.  This is that step written out per Gaussian, following
the reading fixed for this repository (the paper restates none of it):

statistics, per training view, for every Gaussian with a projection (radius > 0):
    grad_accum += || (dL/du * W/2, dL/dv * H/2) ||   (u, v: its projected pixel position)
    denom      += 1
    max_radius  = max(max_radius, radius)

densification step t (every `interval` steps within [start, stop)):
    g      = grad_accum / denom   (0 where denom = 0)
    smax   = max of the three scales exp(log_scale);  o = sigmoid(logit opacity)
    prune  = o < min_opacity  or  (t > reset_interval and (max_radius > max_screen or smax > 0.1 extent))
    dense  = not prune and g >= grad_threshold
    split  = dense and smax >  percent_dense extent
    clone  = dense and smax <= percent_dense extent
    output = [sources that are neither pruned nor split, in index order]
           + [copies of the cloned sources, in index order]
           + [two children per split source, in index order: child k has
              mean = mean + R(q) (s * z[k]), log_scale = log(s / 1.6), all else copied]
    Adam moments: copied for the kept sources, zero for copies and children.

opacity reset (every reset_interval steps): logit opacity = min(logit opacity, logit(0.01)), and the
opacity's Adam moments become 0.

Pruning is decided on the sources; a source that is pruned is neither kept nor cloned nor split.
The random z [n, 2, 3] are inputs.  Parity pins: tests/test_oracle_densify.py.
"""
from __future__ import annotations

import math

import numpy as np

DEFAULTS = dict(grad_threshold=2e-4, percent_dense=0.01, min_opacity=0.005, max_screen=20.0,
                reset_interval=3000, split_n=2, split_shrink=1.6)


def quat_rot(q):
    """Rotation matrix of the normalised quaternion (w, x, y, z) (Hamilton convention)."""
    q = np.asarray(q, np.float64)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def stats(grad_accum, denom, max_radius, dxy, radius, W: int, H: int):
    """One view's statistics (in place on copies; returns the three arrays)."""
    ga, dn, mr = np.array(grad_accum, np.float64), np.array(denom, np.float64), np.array(max_radius, np.float64)
    for i in range(len(radius)):
        if radius[i] > 0:
            ga[i] += math.hypot(dxy[i][0] * W / 2.0, dxy[i][1] * H / 2.0)
            dn[i] += 1.0
            mr[i] = max(mr[i], float(radius[i]))
    return ga, dn, mr


def plan(g, grad_accum, denom, max_radius, step: int, extent: float, cfg=None):
    """Per source: action 0 = prune, 1 = keep, 2 = keep and clone, 3 = split."""
    c = dict(DEFAULTS, **(cfg or {}))
    n = len(g["logit_opacity"])
    act = np.zeros(n, np.int32)
    for i in range(n):
        avg = grad_accum[i] / denom[i] if denom[i] > 0 else 0.0
        smax = max(math.exp(float(s)) for s in g["log_scales"][i])
        o = 1.0 / (1.0 + math.exp(-float(g["logit_opacity"][i])))
        prune = o < c["min_opacity"] or (step > c["reset_interval"] and
                                         (max_radius[i] > c["max_screen"] or smax > 0.1 * extent))
        if prune:
            act[i] = 0
        elif avg >= c["grad_threshold"]:
            act[i] = 3 if smax > c["percent_dense"] * extent else 2
        else:
            act[i] = 1
    return act


def apply(g, m, v, act, z, cfg=None):
    """The output Gaussians and Adam moments (dicts of arrays like `g`) for the actions of `plan`."""
    c = dict(DEFAULTS, **(cfg or {}))
    keys = list(g.keys())
    out = {k: [] for k in keys}
    om = {k: [] for k in keys}
    ov = {k: [] for k in keys}

    def push(src_g, src_m, src_v):
        for k in keys:
            out[k].append(np.asarray(src_g[k], np.float64))
            om[k].append(np.asarray(src_m[k], np.float64))
            ov[k].append(np.asarray(src_v[k], np.float64))

    zero = {k: np.zeros_like(np.asarray(g[k][0], np.float64)) for k in keys}
    n = len(act)
    for i in range(n):  # survivors
        if act[i] in (1, 2):
            push({k: g[k][i] for k in keys}, {k: m[k][i] for k in keys}, {k: v[k][i] for k in keys})
    for i in range(n):  # copies
        if act[i] == 2:
            push({k: g[k][i] for k in keys}, zero, zero)
    for i in range(n):  # children
        if act[i] == 3:
            s = np.exp(np.asarray(g["log_scales"][i], np.float64))
            R = quat_rot(g["quats"][i])
            for k in range(c["split_n"]):
                child = {kk: np.asarray(g[kk][i], np.float64) for kk in keys}
                child["means"] = np.asarray(g["means"][i], np.float64) + R @ (s * np.asarray(z[i][k], np.float64))
                child["log_scales"] = np.log(s / c["split_shrink"])
                push(child, zero, zero)
    stack = lambda d: {k: (np.stack(d[k]) if d[k] else np.zeros((0,) + np.shape(g[k])[1:])) for k in keys}
    return stack(out), stack(om), stack(ov)


def opacity_reset(g, m, v, cap: float = 0.01):
    """logit opacity = min(logit opacity, logit(cap)); the opacity's Adam moments become 0."""
    lim = math.log(cap / (1.0 - cap))
    g = dict(g)
    g["logit_opacity"] = np.minimum(np.asarray(g["logit_opacity"], np.float64), lim)
    m, v = dict(m), dict(v)
    m["logit_opacity"] = np.zeros_like(np.asarray(m["logit_opacity"], np.float64))
    v["logit_opacity"] = np.zeros_like(np.asarray(v["logit_opacity"], np.float64))
    return g, m, v
