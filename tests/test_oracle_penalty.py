"""Pins of the oracle's background-opacity penalty (a variant of the masked loss of Sec. II, "Image
Rendering and Masking": lam x mean of the rendered opacity 1 - T_final over the pixels outside the mask).

* the penalty and its gradient with respect to T_final, by hand with numpy;
* the parameter gradient through the reverse replay (dL/dT_final enters every blended entry's alpha
  term) against the exact dual-number directional derivative of projection + blend + penalty, per
  parameter group and along random tangents, alone and together with the masked loss;
* central finite differences of the penalty on the opacity logits of sampled Gaussians.
"""
import numpy as np
import pytest

import oracle
from tests import scenes

LAM_BG = 0.7
LAM = 0.2


def _scene(n=120, deg=3, seed=11, W=64, H=64):
    g, cams = scenes.random_scene(n, deg, seed, W, H, extent=0.7, log_scale_range=(-3.0, -1.8))
    cam = oracle.camera_block(cams, 0)
    gt, mask = scenes.random_gt(W, H, seed + 100)
    return g, cam, gt, mask


def _penalty_grads(g, cam, bg, mask, dimg=None):
    r = oracle.render(g, cam, bg)
    val, dT = oracle.bg_penalty(r["final_T"], mask, LAM_BG)
    d = np.zeros_like(r["img"]) if dimg is None else dimg
    g2d = oracle.render_backward(g, cam, bg, d, dT)
    return val, oracle.project_backward(g, cam, g2d), r


def test_bg_penalty_by_hand():
    rng = np.random.default_rng(3)
    T = rng.uniform(0.0, 1.0, (17, 23))
    mask = (rng.uniform(0.0, 1.0, T.shape) > 0.4).astype(np.uint8)
    val, dT = oracle.bg_penalty(T, mask, LAM_BG)
    bgp = mask == 0
    assert val == pytest.approx(LAM_BG * float(np.mean(1.0 - T[bgp])), rel=1e-14)
    assert np.all(dT[~bgp] == 0.0)
    assert np.allclose(dT[bgp], -LAM_BG / bgp.sum(), rtol=0, atol=1e-17)
    # no background pixel: no penalty, no gradient
    val, dT = oracle.bg_penalty(T, np.ones_like(mask), LAM_BG)
    assert val == 0.0 and not dT.any()


def test_penalty_grad_vs_dual_tangents():
    g, cam, gt, mask = _scene()
    bg = np.array([0.0, 0.0, 0.0])
    val, grads, _ = _penalty_grads(g, cam, bg, mask)
    assert val > 0.0
    rng = np.random.default_rng(6)
    npar = grads.shape[1]
    # the colour (SH) group has no penalty gradient: T_final does not depend on colour
    assert np.all(grads[:, 14:] == 0.0) and np.abs(grads[:, :11]).max() > 0.0
    groups = [slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11)]
    for gi, sl in enumerate(groups + [slice(0, npar)] * 3):
        tang = np.zeros_like(grads)
        tang[:, sl] = rng.standard_normal(tang[:, sl].shape)
        pv, exact = oracle.penalty_params_dir(g, tang, cam, bg, mask, LAM_BG)
        assert pv == pytest.approx(val, rel=1e-12)
        got = float((grads * tang).sum())
        assert got == pytest.approx(exact, rel=1e-9, abs=1e-14), gi


def test_loss_plus_penalty_grad_vs_dual():
    """Both gradients through one reverse replay equal the sum of the two directional derivatives."""
    g, cam, gt, mask = _scene(seed=21)
    bg = np.array([1.0, 1.0, 1.0])
    r = oracle.render(g, cam, bg)
    _, dimg = oracle.loss(r["img"], gt, mask, LAM, grad=True)
    val, grads, _ = _penalty_grads(g, cam, bg, mask, dimg)
    rng = np.random.default_rng(8)
    for _ in range(3):
        tang = rng.standard_normal(grads.shape)
        _, dl = oracle.loss_params_dir(g, tang, cam, bg, gt, mask, LAM)
        _, dp = oracle.penalty_params_dir(g, tang, cam, bg, mask, LAM_BG)
        assert float((grads * tang).sum()) == pytest.approx(dl + dp, rel=1e-9, abs=1e-14)


def test_penalty_grad_vs_central_fd_on_opacity():
    g, cam, gt, mask = _scene(n=60, seed=31)
    bg = np.array([0.0, 0.0, 0.0])
    _, grads, r = _penalty_grads(g, cam, bg, mask)
    touched = np.flatnonzero(np.abs(grads[:, 10]) > 1e-8)
    assert touched.size >= 5
    h = 1e-5
    for i in touched[:: max(1, touched.size // 8)][:8]:
        vals = []
        for s in (1.0, -1.0):
            v = oracle.flatten_params(g)
            v[i, 10] += s * h
            rr = oracle.render(oracle.unflatten_params(v, 3), cam, bg)
            vals.append(oracle.bg_penalty(rr["final_T"], mask, LAM_BG)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert grads[i, 10] == pytest.approx(fd, rel=1e-5, abs=1e-10), i
