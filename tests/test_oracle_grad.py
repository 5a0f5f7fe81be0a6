"""Pins of the oracle's loss and gradients.

* loss: SSIM(x, x) = 1; closed form on constant images; masked L1 by hand; the masked D-SSIM
  loss against SSIM statistics filtered by scipy (11x11 Gaussian window, zero padding, C1, C2);
* loss gradient: against the dual-number directional derivative and FD;
* parameter gradient (reverse replay + projection Jacobian): against the
  exact dual-number directional derivative of the whole pipeline, along
  random tangents and per parameter group, and against central finite
  differences (h = 1e-4) on every parameter of sampled Gaussians.
"""
import math

import numpy as np
import pytest

import oracle
from tests import scenes

LAM = 0.2


def test_masked_l1_by_hand():
    img = np.zeros((3, 2, 2))
    gt = np.zeros((3, 2, 2))
    img[0, 0, 0] = 0.5
    img[1, 0, 1] = -0.25
    img[2, 1, 1] = 1.0  # masked out
    mask = np.array([[1, 1], [1, 0]], np.uint8)
    val, d = oracle.loss(img, gt, mask, 0.0)
    assert val == pytest.approx((0.5 + 0.25) / (3 * 3))
    assert d[0, 0, 0] == pytest.approx(1 / 9) and d[1, 0, 1] == pytest.approx(-1 / 9)
    assert d[2, 1, 1] == 0 and d[0, 1, 0] == 0  # masked; and sign(0) = 0
    assert oracle.loss(img, gt, np.zeros((2, 2), np.uint8), 0.0)[0] == 0.0


def test_ssim_identity_and_constant_closed_form():
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (3, 30, 40))
    mask = np.ones((30, 40), np.uint8)
    assert oracle.loss(x, x, mask, 1.0, grad=False) == pytest.approx(0.0, abs=1e-12)
    # constant images c1, c2: interior pixels (window fully inside) have sigma = 0 and
    # SSIM = (2 c1 c2 + C1) / (c1^2 + c2^2 + C1)
    c1, c2 = 0.3, 0.8
    a = np.full((3, 30, 40), c1)
    b = np.full((3, 30, 40), c2)
    inner = np.zeros((30, 40), np.uint8)
    inner[5:-5, 5:-5] = 1
    C1 = 0.01 ** 2
    ssim = (2 * c1 * c2 + C1) / (c1 ** 2 + c2 ** 2 + C1)
    assert oracle.loss(a, b, inner, 1.0, grad=False) == pytest.approx(1 - ssim, rel=1e-12)


@pytest.mark.parametrize("lam", [0.0, 0.2, 1.0])
def test_loss_grad_vs_dual_and_fd(lam):
    rng = np.random.default_rng(1)
    H, W = 23, 37
    img = rng.uniform(0, 1, (3, H, W))
    gt = rng.uniform(0, 1, (3, H, W))
    mask = (rng.uniform(0, 1, (H, W)) > 0.3).astype(np.uint8)
    val, d = oracle.loss(img, gt, mask, lam)
    for k in range(5):
        direction = rng.standard_normal(img.shape)
        exact = oracle.loss_dir(img, direction, gt, mask, lam)
        assert float((d * direction).sum()) == pytest.approx(exact, rel=1e-10, abs=1e-14)
        h = 1e-6
        fd = (oracle.loss(img + h * direction, gt, mask, lam, grad=False)
              - oracle.loss(img - h * direction, gt, mask, lam, grad=False)) / (2 * h)
        # |C - G| kinks are far from every pixel here, so FD is smooth
        assert fd == pytest.approx(exact, rel=1e-5)


def _scene(n=120, deg=3, seed=11, W=64, H=64):
    g, cams = scenes.random_scene(n, deg, seed, W, H, extent=0.7, log_scale_range=(-3.0, -1.8))
    cam = oracle.camera_block(cams, 0)
    gt, mask = scenes.random_gt(W, H, seed + 100)
    return g, cam, gt, mask


def test_param_grad_vs_dual_random_tangents():
    g, cam, gt, mask = _scene()
    bg = np.array([1.0, 1.0, 1.0])
    r = oracle.loss_and_grads(g, cam, bg, gt, mask, LAM)
    grads = r["grads"]
    rng = np.random.default_rng(5)
    npar = grads.shape[1]
    groups = [slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11), slice(11, 14), slice(14, npar)]
    for gi, sl in enumerate(groups + [slice(0, npar)] * 3):
        tang = np.zeros_like(grads)
        tang[:, sl] = rng.standard_normal(tang[:, sl].shape)
        val, exact = oracle.loss_params_dir(g, tang, cam, bg, gt, mask, LAM)
        assert val == pytest.approx(r["loss"], rel=1e-12)
        got = float((grads * tang).sum())
        assert got == pytest.approx(exact, rel=1e-9, abs=1e-14), gi


def _flips(g, cam, i, k, h):
    """Whether perturbing parameter k of Gaussian i by +-h changes any discrete decision."""
    base = oracle.render(g, cam, np.ones(3))
    out = []
    flat = oracle.flatten_params(g)
    deg = int(round(math.sqrt(g["sh"].reshape(len(flat), -1).shape[1] // 3))) - 1
    for s in (+1, -1):
        f2 = flat.copy()
        f2[i, k] += s * h
        gg = oracle.unflatten_params(f2, deg)
        p0 = oracle.project(g, cam)
        p1 = oracle.project(gg, cam)
        rr = oracle.render(gg, cam, np.ones(3))
        changed = (p0["radius"][i] != p1["radius"][i] or np.any(p0["rect"][i] != p1["rect"][i])
                   or p0["clamp"][i] != p1["clamp"][i]
                   or not np.array_equal(base["n_contrib"], rr["n_contrib"]))
        out.append(changed)
    return any(out)


def test_param_grad_vs_central_fd():
    """Central FD (h = 1e-4) of the FP64 loss on every parameter of sampled Gaussians; parameters whose
    perturbation flips a discrete decision (cull, rectangle, clamp, skip/stop pattern) are excluded."""
    g, cam, gt, mask = _scene(n=60, seed=12, W=48, H=48)
    bg = np.ones(3)
    r = oracle.loss_and_grads(g, cam, bg, gt, mask, LAM)
    grads = r["grads"]
    flat = oracle.flatten_params(g)
    deg = 3
    h = 1e-4
    vis = np.nonzero(oracle.project(g, cam)["radius"] > 0)[0]
    rng = np.random.default_rng(0)
    sample = rng.choice(vis, size=min(6, len(vis)), replace=False)
    checked = excluded = 0
    for i in sample:
        for k in range(flat.shape[1]):
            if _flips(g, cam, i, k, h):
                excluded += 1
                continue
            vals = []
            for s in (+1, -1):
                f2 = flat.copy()
                f2[i, k] += s * h
                rr = oracle.render(oracle.unflatten_params(f2, deg), cam, bg)
                vals.append(oracle.loss(rr["img"], gt, mask, LAM, grad=False))
            fd = (vals[0] - vals[1]) / (2 * h)
            scale = np.abs(grads[i]).max() + 1e-12
            assert abs(fd - grads[i, k]) <= 1e-4 * scale + 1e-7 * abs(fd), (i, k, fd, grads[i, k])
            checked += 1
    assert checked >= 0.8 * (checked + excluded)


def test_alpha_clamp_gradient_is_zero():
    """A splat whose alpha is clamped at 0.99 everywhere it is seen gets no opacity gradient."""
    W, H = 16, 16
    cams = scenes.identity_camera(W, H)
    cam = oracle.camera_block(cams, 0)
    # screen sigma ~ 80 px, so o G > 0.99 on the whole 16 x 16 image
    g = dict(means=np.array([[0.0, 0.0, 2.0]]), log_scales=np.full((1, 3), math.log(12.0)),
             quats=np.array([[1.0, 0, 0, 0]]), logit_opacity=np.array([40.0]),
             sh=np.zeros((1, 1, 3)))
    gt = np.zeros((3, H, W))
    mask = np.ones((H, W), np.uint8)
    r = oracle.loss_and_grads(g, cam, np.ones(3), gt, mask, 0.0)
    assert r["g2d"]["dopacity"][0] == 0.0 and np.all(r["g2d"]["dconic"][0] == 0.0)
    assert np.abs(r["g2d"]["drgb"][0]).max() > 0


def test_masked_ssim_loss_matches_library_filtered_statistics():
    """The loss at lambda = 0.2 against SSIM statistics from scipy's Gaussian filter (sigma 1.5, radius 5,
    zero padding: the 11x11 window), C1 = 0.01^2, C2 = 0.03^2, masked means over mask pixels and channels."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(5)
    H, W = 29, 41
    x = rng.uniform(0, 1, (3, H, W))
    y = np.clip(0.7 * x + rng.normal(0, 0.1, (3, H, W)), 0, 1)
    mask = (rng.uniform(0, 1, (H, W)) > 0.25).astype(np.uint8)

    def g(a):
        return ndimage.gaussian_filter(a, 1.5, mode="constant", cval=0.0, truncate=5.0 / 1.5)

    C1, C2 = 0.01 ** 2, 0.03 ** 2
    ssim = []
    for c in range(3):
        mx, my = g(x[c]), g(y[c])
        sxx, syy, sxy = g(x[c] * x[c]) - mx * mx, g(y[c] * y[c]) - my * my, g(x[c] * y[c]) - mx * my
        ssim.append(((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2)))
    m = mask.astype(bool)
    ssim_mean = np.mean([s[m] for s in ssim])
    l1 = np.abs(x - y)[:, m].mean()
    expected = 0.8 * l1 + 0.2 * (1.0 - ssim_mean)
    assert oracle.loss(x, y, mask, 0.2, grad=False) == pytest.approx(expected, rel=1e-10)
