"""CUDA path vs the FP64 oracle, element by element (needs a GPU).

Bars (from the method's statement of parity):
* visibility, radius, tile rectangle and tile count of every Gaussian: equal,
  except decisions the oracle flags as float32 near-ties (its stated error
  model), whose count must stay at or below 1e-5 of the instances;
* sorted per-tile lists: equal to the oracle's own lists (its FP64 projection,
  depth key = float32 rounding of the FP64 camera-space z), except tiles that
  hold such a flagged Gaussian, counted the same way;
* images: max abs error <= 1e-4 per colour channel, excluding pixels whose
  FP64 decisions sit within 1e-5 (relative) of a threshold and tiles touched by
  a flagged Gaussian whose decisions differ (counted, < 1% of the image);
* gradients: per parameter group, max |g_gpu - g_orc| <= 1e-3 * max |g_orc|.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import scenes
from tests.gpu_util import discrete_mismatch, exclusion_mask, gauss64, rects, run_gpu

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4
GRAD_TOL = 1e-3
BG = np.array([1.0, 1.0, 1.0])


def _case(n, deg, seed, W, H, extent=0.9, ls=(-3.5, -2.0)):
    g, cams = scenes.random_scene(n, deg, seed, W, H, extent=extent, log_scale_range=ls)
    return g, cams


PREPROCESS_CASES = [(3000, 3, 200, 150, 0), (2000, 0, 128, 128, 1), (1500, 1, 97, 61, 2), (2500, 2, 256, 144, 3)]


@pytest.mark.parametrize("n,deg,W,H,seed", PREPROCESS_CASES)
def test_preprocess_parity(n, deg, W, H, seed):
    g, cams = _case(n, deg, seed, W, H)
    out = run_gpu(g, cams, deg, BG)
    cam = oracle.camera_block(cams, 0)
    o = oracle.project(gauss64(g), cam)
    # discrete decisions: every difference is a near-tie the oracle flags, and they are rare
    mism, flagged = discrete_mismatch(o, out["xy4"], out["radius"], out["tiles"], W, H)
    n_inst = int(o["tiles"].sum())
    print(f"preprocess n={n}: {int(mism.sum())} differing decisions (all flagged: {flagged}), "
          f"{int((o['unstable'] != 0).sum())} flagged Gaussians, {n_inst} instances")
    assert flagged, np.nonzero(mism)[0][:10]
    assert mism.sum() <= 1e-5 * n_inst
    # the sort key: the correctly rounded float32 camera-space z on both sides
    assert np.array_equal(out["depth"], o["depth"].astype(np.float32))
    both = (o["radius"] > 0) & (out["radius"] > 0)
    # pixel position: float pairs, ~2^-44 relative
    assert np.allclose(out["xy"][both], o["xy"][both], rtol=1e-11, atol=1e-9)
    A = o["conic"][both]
    sc = np.abs(A).max(axis=1, keepdims=True)
    assert np.all(np.abs(out["conic_op"][both, :3] - A) <= 2e-4 * sc)
    assert np.allclose(out["conic_op"][both, 3], o["opacity"][both], rtol=1e-5, atol=1e-6)
    assert np.allclose(out["rgb"][both, :3], o["rgb"][both], atol=2e-5)


def _lists_vs_oracle(out, o, W, H):
    """Tiles whose GPU list differs from the oracle's own list; each must hold a Gaussian with a flagged
    decision that differs between the two sides.  Returns (differing tiles, instances in them)."""
    L = oracle.bin_sort(o["xy"], o["radius"], o["depth"], W, H)
    mism, flagged = discrete_mismatch(o, out["xy4"], out["radius"], out["tiles"], W, H)
    assert flagged
    bad = set(np.nonzero(mism)[0].tolist())
    n_bad, inst_bad = 0, 0
    for t in range(L["ranges"].shape[0]):
        a, b = out["ranges"][t]
        oa, ob = L["ranges"][t]
        gl, ol = out["vals"][a:b], L["idx"][oa:ob]
        if len(gl) == len(ol) and np.array_equal(gl, ol):
            continue
        assert bad & (set(gl.tolist()) ^ set(ol.tolist())), f"tile {t} differs without a flagged Gaussian"
        n_bad += 1
        inst_bad += max(len(gl), len(ol))
    return n_bad, inst_bad, len(L["idx"])


@pytest.mark.parametrize("n,deg,W,H,seed", [(3000, 3, 200, 150, 4), (5000, 0, 333, 97, 5)])
def test_sort_lists_bit_exact(n, deg, W, H, seed):
    """The GPU's sorted tile lists equal the oracle's lists from its own FP64 projection (depth key: the
    float32 rounding of the FP64 camera-space z; equal keys by Gaussian index), tile by tile."""
    g, cams = _case(n, deg, seed, W, H)
    out = run_gpu(g, cams, deg, BG)
    assert out["status"] == 0
    assert len(out["vals"]) == int(out["tiles"].sum())
    o = oracle.project(gauss64(g), oracle.camera_block(cams, 0))
    n_bad, inst_bad, I = _lists_vs_oracle(out, o, W, H)
    print(f"lists: {n_bad} tiles ({inst_bad} instances) differ at flagged near-ties, of {I} instances")
    assert inst_bad <= 1e-5 * I


@pytest.mark.parametrize("n,deg,W,H,seed", [(3000, 3, 200, 150, 6), (800, 0, 64, 64, 7), (4000, 1, 161, 93, 8)])
def test_render_parity(n, deg, W, H, seed):
    g, cams = _case(n, deg, seed, W, H)
    bg = np.array([0.2, 0.5, 0.9])
    out = run_gpu(g, cams, deg, bg)
    cam = oracle.camera_block(cams, 0)
    o = oracle.render(gauss64(g), cam, bg)
    op = oracle.project(gauss64(g), cam)
    excl, ndiff, flagged = exclusion_mask(op, out["xy4"], out["radius"], out["tiles"], o["margin"], W, H)
    print(f"render n={n}: {excl.sum()} of {excl.size} pixels excluded ({ndiff} flagged Gaussians differ)")
    assert flagged and excl.mean() < 0.01, (excl.mean(), ndiff)
    err = np.abs(out["img"][0] - o["img"]).max(axis=0)
    assert err[~excl].max() <= IMG_TOL, err[~excl].max()
    assert np.abs(out["final_T"][0] - o["final_T"])[~excl].max() <= IMG_TOL
    assert np.array_equal(out["n_contrib"][0][~excl], o["n_contrib"][~excl])


@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_loss_parity(lam):
    W, H = 150, 110
    rng = np.random.default_rng(3)
    img = rng.uniform(0, 1, (1, 3, H, W)).astype(np.float32)
    gt, mask = scenes.random_gt(W, H, 9)
    import paper_2509_12138_gb300 as gsp
    fr = gsp.Frame(1, gsp.Units.single(1), W, H, 0, with_backward=False)
    fr.img.copy_(torch.from_numpy(img))
    fr.loss(torch.from_numpy(gt).cuda(), torch.from_numpy(mask).cuda(), lam)
    val, d = oracle.loss(img[0].astype(np.float64), gt.astype(np.float64), mask, lam)
    assert float(fr.loss_val.item()) == pytest.approx(val, rel=1e-5)
    dg = fr.dimg.cpu().numpy()[0]
    assert np.abs(dg - d).max() <= 1e-3 * np.abs(d).max()


@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_loss_parity_sparse_mask(lam):
    """A mask covering a disc and a thin stripe only: most 16x16 tiles hold no mask pixel and many gradient
    windows reach none, so the SSIM kernels' tile skipping is exercised; loss and gradient still match the
    oracle, and the gradient is exactly zero wherever no mask pixel lies within the window's reach."""
    W, H = 200, 150
    rng = np.random.default_rng(4)
    img = rng.uniform(0, 1, (1, 3, H, W)).astype(np.float32)
    gt, _ = scenes.random_gt(W, H, 10)
    yy, xx = np.mgrid[0:H, 0:W]
    mask = (((xx - 60) ** 2 + (yy - 50) ** 2 < 25 ** 2) | ((yy >= 120) & (yy < 122) & (xx > 100))).astype(np.uint8)
    import paper_2509_12138_gb300 as gsp
    fr = gsp.Frame(1, gsp.Units.single(1), W, H, 0, with_backward=False)
    fr.img.copy_(torch.from_numpy(img))
    fr.loss(torch.from_numpy(gt).cuda(), torch.from_numpy(mask).cuda(), lam)
    val, d = oracle.loss(img[0].astype(np.float64), gt.astype(np.float64), mask, lam)
    assert float(fr.loss_val.item()) == pytest.approx(val, rel=1e-5)
    dg = fr.dimg.cpu().numpy()[0]
    assert np.abs(dg - d).max() <= 1e-3 * np.abs(d).max()
    far = np.ones((H, W), bool)
    for y, x in zip(*np.nonzero(mask)):
        far[max(0, y - 5):y + 6, max(0, x - 5):x + 6] = False
    assert far.mean() > 0.5 and np.all(dg[:, far] == 0.0)


def _group_check(gg, go, deg, tol=GRAD_TOL):
    groups = dict(mean=slice(0, 3), log_scale=slice(3, 6), quat=slice(6, 10), opacity=slice(10, 11),
                  sh_dc=slice(11, 14), sh_rest=slice(14, gg.shape[1]))
    if deg == 0:
        groups.pop("sh_rest")
    for name, sl in groups.items():
        ref = go[:, sl]
        scale = np.abs(ref).max()
        if scale == 0:
            continue
        err = np.abs(gg[:, sl] - ref).max()
        assert err <= tol * scale, (name, err, scale)


@pytest.mark.parametrize("n,deg,W,H,seed,lam", [(500, 3, 64, 64, 10, 0.2), (2000, 3, 150, 100, 11, 0.2),
                                                (1500, 0, 128, 128, 12, 0.0), (1200, 1, 90, 70, 13, 0.2)])
def test_backward_parity(n, deg, W, H, seed, lam):
    """All parameter gradients of the full pipeline (loss -> blend bwd -> projection bwd)."""
    g, cams = _case(n, deg, seed, W, H, ls=(-3.0, -1.8))
    gt, mask = scenes.random_gt(W, H, seed + 50)
    out = run_gpu(g, cams, deg, BG, gt[None], mask[None], lam)
    cam = oracle.camera_block(cams, 0)
    r = oracle.loss_and_grads(gauss64(g), cam, BG, gt.astype(np.float64), mask, lam)
    assert out["loss"] == pytest.approx(r["loss"], rel=1e-4)
    # screen-space gradients
    g2 = r["g2d"]
    vis = out["radius"] > 0
    for a, b in [(out["dxy"][:, :2], g2["dxy"]), (out["dco"][:, :3], g2["dconic"]), (out["dco"][:, 3], g2["dopacity"]),
                 (out["drgb"][:, :3], g2["drgb"])]:
        sc = np.abs(b).max()
        assert np.abs(a[vis] - b[vis]).max() <= GRAD_TOL * sc
    _group_check(out["grads"], r["grads"], deg)


def test_multi_unit_batch_parity():
    """Three views of one scene in one launch chain: each unit equals its own single-view oracle run."""
    n, deg = 1500, 3
    g = synth.random_gaussians(n, deg, 20, extent=0.7, log_scale_range=(-3.2, -2.0))
    cams = synth.orbital_cameras(3, 3.0, width=120, height=88)
    gts = np.stack([scenes.random_gt(120, 88, 30 + k)[0] for k in range(3)])
    masks = np.stack([scenes.random_gt(120, 88, 30 + k)[1] for k in range(3)])
    out = run_gpu(g, cams, deg, BG, gts, masks, 0.2)
    loss_sum = 0.0
    grad_sum = None
    for k in range(3):
        cam = oracle.camera_block(cams, k)
        o = oracle.render(gauss64(g), cam, BG)
        op = oracle.project(gauss64(g), cam)
        P = slice(k * n, (k + 1) * n)
        excl, _, flagged = exclusion_mask(op, out["xy4"][P], out["radius"][P], out["tiles"][P], o["margin"], 120, 88)
        assert flagged and excl.mean() < 0.01
        assert np.abs(out["img"][k] - o["img"]).max(axis=0)[~excl].max() <= IMG_TOL
        r = oracle.loss_and_grads(gauss64(g), cam, BG, gts[k].astype(np.float64), masks[k], 0.2)
        loss_sum += r["loss"]
        grad_sum = r["grads"] if grad_sum is None else grad_sum + r["grads"]
    # loss and gradients are the mean over units
    assert out["loss"] == pytest.approx(loss_sum / 3, rel=1e-4)
    _group_check(out["grads"], grad_sum / 3, deg)


def test_adam_parity():
    import paper_2509_12138_gb300 as gsp
    n, deg = 1000, 3
    g = synth.random_gaussians(n, deg, 40)
    params = gsp.pack_params(g, deg)
    opt = gsp.Adam(params, deg, extent=2.0, lr_steps=10)
    rng = np.random.default_rng(0)
    p_ref = params.cpu().numpy().astype(np.float64).reshape(-1)
    m_ref = np.zeros_like(p_ref)
    v_ref = np.zeros_like(p_ref)
    npl = params.shape[0]
    for t in range(1, 6):
        grads = torch.from_numpy(rng.standard_normal(params.shape).astype(np.float32)).cuda()
        gnp = grads.cpu().numpy().astype(np.float64).reshape(-1)
        frac = min(t, 10) / 10
        lr = opt.lr_init.astype(np.float64) * (opt.lr_final.astype(np.float64) /
                                               np.where(opt.lr_init > 0, opt.lr_init, 1)) ** frac
        lr = np.where(opt.lr_init == opt.lr_final, opt.lr_init, lr)
        lr_el = np.repeat(lr.reshape(npl, 1, 4), n, axis=1).reshape(-1)
        p_ref, m_ref, v_ref = oracle.adam(p_ref, gnp, m_ref, v_ref, lr_el, 0.9, 0.999, 1e-15, t)
        opt.step(grads, zero_grad=True)
        assert torch.count_nonzero(grads).item() == 0
    got = params.cpu().numpy().astype(np.float64).reshape(-1)
    assert np.allclose(got, p_ref, rtol=1e-5, atol=1e-6)
    assert np.allclose(opt.m.cpu().numpy().reshape(-1), m_ref, rtol=1e-4, atol=1e-7)
    assert int(opt.step_dev.item()) == 5


def test_autograd_function_matches_frame_backward():
    import paper_2509_12138_gb300 as gsp
    n, deg, W, H = 800, 1, 80, 64
    g, cams = _case(n, deg, 50, W, H)
    params = gsp.pack_params(g, deg).requires_grad_(True)
    fr = gsp.Frame(n, gsp.Units.single(n), W, H, deg)
    camd = gsp.pack_cameras(cams)
    img = gsp.rasterize(params, fr, camd, BG)
    w = torch.from_numpy(np.random.default_rng(51).standard_normal(tuple(img.shape)).astype(np.float32)).cuda()
    (img * w).sum().backward()
    fr2 = gsp.Frame(n, gsp.Units.single(n), W, H, deg)
    fr2.forward(params.detach(), camd, BG)
    g2 = fr2.backward(params.detach(), camd, BG, w.contiguous())
    # the same kernels on both paths: equal up to the order of the float atomics that accumulate gradients
    assert torch.allclose(params.grad, g2, rtol=1e-4, atol=1e-5 * float(g2.abs().max()))
    # and against the oracle: d<w, img>/dparams
    cam = oracle.camera_block(cams, 0)
    d2 = oracle.render_backward(gauss64(g), cam, BG, w[0].cpu().numpy().astype(np.float64))
    go = oracle.project_backward(gauss64(g), cam, d2)
    _group_check(gsp.unpack_grads(params.grad, deg), go, deg)


# ---------------------------------------------------------------- edge cases
def test_empty_and_all_culled():
    import paper_2509_12138_gb300 as gsp
    W, H = 40, 30
    cams = scenes.identity_camera(W, H)
    g = synth.random_gaussians(50, 0, 60, center=(0, 0, -5.0), extent=0.5)  # all behind the camera
    out = run_gpu(g, cams, 0, BG)
    assert np.all(out["radius"] == 0) and len(out["vals"]) == 0
    assert np.allclose(out["img"], 1.0) and np.all(out["final_T"] == 1.0) and np.all(out["n_contrib"] == 0)
    # zero Gaussians
    fr = gsp.Frame(0, gsp.Units.single(0), W, H, 0)
    fr.forward(torch.zeros((4, 0, 4), device="cuda"), gsp.pack_cameras(cams), BG)
    torch.cuda.synchronize()
    assert np.allclose(fr.img.cpu().numpy(), 1.0)


def test_capacity_overflow_sets_status_without_fault():
    g, cams = _case(2000, 0, 70, 128, 96)
    out = run_gpu(g, cams, 0, BG, max_instances=100)
    assert out["status"] & 2  # GS_ERR_CAPACITY
    assert len(out["vals"]) == 100


def test_invalid_arguments_rejected_on_host():
    import ctypes as C
    from paper_2509_12138_gb300 import _lib
    L = _lib.load()
    assert L.gs_param_planes(4) == -1 and L.gs_param_planes(3) == 15 and L.gs_param_planes(0) == 4
    rc = L.gs_preprocess(None, 10, 0, None, None, 10, 10, None, None, None, None)
    assert rc == 1


def test_blend_work_counters():
    """The diagnostic counters: the reverse replay's unit is sum(n_contrib); every blended pair lies before
    n_contrib, and the forward walk evaluates at least the entries up to n_contrib."""
    import paper_2509_12138_gb300 as gsp
    n, deg, W, H = 1500, 1, 120, 90
    g, cams = _case(n, deg, 71, W, H)
    params = gsp.pack_params(g, deg)
    camd = gsp.pack_cameras(cams)
    fr = gsp.Frame(n, gsp.Units.single(n), W, H, deg, with_backward=False, with_loss=False)
    fr.fit_capacity(params, camd)
    fr.forward(params, camd, BG)
    c = fr.blend_pairs()
    nc = int(fr.n_contrib.sum().item())
    assert c["bwd_pairs"] == nc > 0
    assert 0 < c["blended"] <= c["bwd_pairs"] <= c["fwd_pairs"]
    # a blended pair has alpha >= 1/255, so its record's alpha box (and block mask) reaches the pixel
    assert c["blended"] <= c["bwd_pairs_masked"] <= c["bwd_pairs"]
    assert c["bwd_pairs_masked"] <= c["fwd_pairs_masked"] <= c["fwd_pairs"]
    assert c["fwd_pairs_masked"] < c["fwd_pairs"]
    lens = (fr.ranges[:, 1] - fr.ranges[:, 0]).cpu().numpy()
    assert c["fwd_pairs"] <= int(lens.sum()) * 256


def test_fused_projection_backward_adam_vs_oracle():
    """The fused projection backward + Adam kernel the benchmark runs, against the oracle's FP64 parameter
    gradient (reverse replay, dual-number projection Jacobian) followed by the oracle's Adam step.  The
    moments start from seeded values in the range training reaches (so the update depends smoothly on the
    gradient) at step t = 11 of a log-linear learning-rate schedule."""
    import paper_2509_12138_gb300 as gsp
    n, deg, W, H, seed = 1200, 3, 120, 90, 15
    g, cams = _case(n, deg, seed, W, H, ls=(-3.0, -1.8))
    gt, mask = scenes.random_gt(W, H, seed + 50)
    cam = oracle.camera_block(cams, 0)
    r = oracle.loss_and_grads(gauss64(g), cam, BG, gt.astype(np.float64), mask, 0.2)
    go = r["grads"]
    groups = [slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11), slice(11, 14), slice(14, go.shape[1])]
    sc = np.zeros(go.shape[1])
    for sl in groups:
        sc[sl] = np.abs(go[:, sl]).max()
    rng = np.random.default_rng(seed)
    m0 = rng.normal(0.0, 1.0, go.shape) * sc
    v0 = rng.uniform(0.5, 2.0, go.shape) * sc * sc
    fr = gsp.Frame(n, gsp.Units.single(n), W, H, deg)
    params = gsp.pack_params(g, deg)
    camd = gsp.pack_cameras(cams)
    fr.fit_capacity(params, camd)
    fr.forward(params, camd, BG)
    fr.loss(torch.from_numpy(gt).cuda()[None], torch.from_numpy(mask).cuda()[None], 0.2)
    fr.blend_backward(BG)
    opt = gsp.Adam(params, deg, extent=1.0, lr_steps=100)
    opt.m.copy_(gsp.pack_params(oracle.unflatten_params(m0, deg), deg))
    opt.v.copy_(gsp.pack_params(oracle.unflatten_params(v0, deg), deg))
    opt.step_dev.fill_(10)
    opt.fused_step(fr, camd, keep_grads=True)
    torch.cuda.synchronize()
    assert fr.read_status() == 0
    # the gradient the fused kernel formed
    _group_check(gsp.unpack_grads(fr.grads, deg), go, deg)
    # Adam at t = 11 with the per-element learning rates of the schedule
    t, steps = 11, 100
    li, lf = opt.lr_init.astype(np.float64), opt.lr_final.astype(np.float64)
    lr = np.where(li == lf, li, li * (lf / np.where(li > 0, li, 1.0)) ** (min(t, steps) / steps))
    npl = params.shape[0]
    lr_el = gsp.unpack_grads(torch.from_numpy(np.repeat(lr.reshape(npl, 1, 4), n, axis=1).astype(np.float32)), deg)
    p0 = oracle.flatten_params(gsp.unpack_params(gsp.pack_params(g, deg), deg))
    p_ref, m_ref, v_ref = oracle.adam(p0, go, m0, v0, lr_el.astype(np.float64), 0.9, 0.999, 1e-15, t)
    p_gpu = oracle.flatten_params(gsp.unpack_params(params, deg))
    m_gpu = gsp.unpack_grads(opt.m, deg)
    v_gpu = gsp.unpack_grads(opt.v, deg)
    # a gradient error of 1e-3 of the group scale moves m by 1e-4 of it, v by ~1e-3 of its own size, and the
    # update by ~2e-4 of the learning rate; on top of float32 rounding of each stored value
    ulp = lambda x: np.spacing(np.abs(x).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(m_gpu - m_ref) <= 1e-4 * sc + 4 * ulp(m_ref))
    assert np.all(np.abs(v_gpu - v_ref) <= 3e-3 * np.abs(v_ref) + 4 * ulp(v_ref))
    assert np.all(np.abs(p_gpu - p_ref) <= 1e-3 * lr_el + 4 * ulp(p_ref))
    assert int(opt.step_dev.item()) == 11


def test_sparse_adam_skips_only_gaussians_without_gradient():
    """With the sparse flag, a Gaussian whose screen-space gradient is zero in the step (here: behind the
    image, or outside the loss mask) keeps its parameters and moments; every other Gaussian gets exactly
    the dense update."""
    import paper_2509_12138_gb300 as gsp
    n, deg, W, H = 1500, 1, 96, 72
    g, cams = _case(n, deg, 30, W, H)
    g["means"][:200, 0] += 50.0  # far to the side of the view: culled, no gradient
    gt, mask = scenes.random_gt(W, H, 31)
    rng = np.random.default_rng(1)
    res = []
    for sparse in (False, True):
        # fixed-point gradient accumulation: both runs see bit-identical screen-space gradients
        fr = gsp.Frame(n, gsp.Units.single(n), W, H, deg, deterministic=True)
        params = gsp.pack_params(g, deg)
        camd = gsp.pack_cameras(cams)
        fr.fit_capacity(params, camd)
        fr.forward(params, camd, BG)
        fr.loss(torch.from_numpy(gt).cuda()[None], torch.from_numpy(mask).cuda()[None], 0.2)
        fr.blend_backward(BG)
        opt = gsp.Adam(params, deg, extent=1.0, lr_steps=100)
        r = np.random.default_rng(1)
        opt.m.copy_(torch.from_numpy(r.normal(0, 1e-3, tuple(opt.m.shape)).astype(np.float32)))
        opt.v.copy_(torch.from_numpy(r.uniform(1e-7, 1e-6, tuple(opt.v.shape)).astype(np.float32)))
        opt.step_dev.fill_(4)
        m0, v0, p0 = opt.m.clone(), opt.v.clone(), params.clone()
        opt.sparse = sparse
        opt.fused_step(fr, camd, keep_grads=True)
        torch.cuda.synchronize()
        assert fr.read_status() == 0
        g2 = torch.cat([fr.dxy[:n].abs(), fr.dco[:n].abs(), fr.drgb[:n, :3].abs()], 1).sum(1) > 0
        res.append(dict(p=params.clone(), m=opt.m.clone(), v=opt.v.clone(), p0=p0, m0=m0, v0=v0, touched=g2))
    dense, sp = res
    touched = sp["touched"]
    assert torch.equal(touched, dense["touched"]) and 0 < int(touched.sum()) < n
    assert int((~touched[:200]).sum()) == 200
    for k in ("p", "m", "v"):
        # touched Gaussians: the dense update bit for bit; untouched: unchanged state
        assert torch.equal(sp[k][:, touched], dense[k][:, touched]), k
        assert torch.equal(sp[k][:, ~touched], sp[k + "0"][:, ~touched]), k
    # the dense step does move untouched Gaussians (momentum), so the two differ there
    assert not torch.equal(dense["p"][:, ~touched], dense["p0"][:, ~touched])


@pytest.mark.parametrize("sparse", [False, True])
def test_fused_next_projection_equals_separate_preprocess(sparse):
    """gs_project_bwd_adam_next: the same update as gs_project_bwd_adam (parameters and moments bit for bit),
    and over the frame's records exactly what gs_preprocess writes for the updated parameters and the next
    camera (position pairs, conics, colours, depths, radii, tile counts)."""
    import paper_2509_12138_gb300 as gsp
    n, deg, W, H = 3000, 3, 160, 120
    g = synth.random_gaussians(n, deg, 41, extent=0.8, log_scale_range=(-3.5, -2.0))
    cams = synth.orbital_cameras(2, 3.0, width=W, height=H)
    camd = gsp.pack_cameras(cams)
    cam_a, cam_b = camd[0:96], camd[96:192]
    gt, mask = scenes.random_gt(W, H, 42)
    fr = gsp.Frame(n, gsp.Units.single(n), W, H, deg, deterministic=True)
    params = gsp.pack_params(g, deg)
    fr.fit_capacity(params, cam_a)
    fr.forward(params, cam_a, BG)
    fr.loss(torch.from_numpy(gt).cuda()[None], torch.from_numpy(mask).cuda()[None], 0.2)
    fr.blend_backward(BG)
    opt = gsp.Adam(params, deg, extent=1.0, lr_steps=100)
    opt.sparse = sparse
    r = np.random.default_rng(3)
    m0 = torch.from_numpy(r.normal(0, 1e-3, tuple(opt.m.shape)).astype(np.float32)).cuda()
    v0 = torch.from_numpy(r.uniform(1e-7, 1e-6, tuple(opt.v.shape)).astype(np.float32)).cuda()
    p0 = params.clone()
    recs = ("xy", "conic_op", "rgb", "depth", "radius", "tiles")
    out = []
    for fused in (False, True):
        params.copy_(p0)
        opt.m.copy_(m0)
        opt.v.copy_(v0)
        opt.step_dev.fill_(2)
        fr.preprocess(params, cam_a)  # this step's records (the fused kernel reads their radii)
        if fused:
            opt.fused_step(fr, cam_a, next_cams_dev=cam_b)
        else:
            opt.fused_step(fr, cam_a)
            fr.preprocess(params, cam_b)
        torch.cuda.synchronize()
        assert fr.read_status() == 0
        out.append({k: getattr(fr, k)[:n].clone() for k in recs} | dict(p=params.clone(), m=opt.m.clone(),
                                                                          v=opt.v.clone()))
    a, b = out
    for k in ("p", "m", "v"):
        assert torch.equal(a[k], b[k]), k
    vis = a["radius"] > 0
    assert int(vis.sum()) > n // 2
    for k in ("depth", "radius", "tiles"):
        assert torch.equal(a[k], b[k]), k
    for k in ("xy", "conic_op", "rgb"):  # written for visible records only
        assert torch.equal(a[k][vis], b[k][vis]), k



def test_fused_next_projection_two_units():
    """Two disjoint units (two partitions, each with its own camera now and its own next camera): the update
    and every record equal gs_project_bwd_adam followed by gs_preprocess of the updated parameters for that
    unit's next camera."""
    import paper_2509_12138_gb300 as gsp
    n, deg, W, H = 4000, 1, 128, 96
    g = synth.random_gaussians(n, deg, 51, extent=0.8, log_scale_range=(-3.5, -2.0))
    camd = gsp.pack_cameras(synth.orbital_cameras(4, 3.0, width=W, height=H))
    now, nxt = torch.cat([camd[0:96], camd[96:192]]), torch.cat([camd[192:288], camd[288:384]])
    units = gsp.Units(np.array([0, 2500], np.int64), np.array([2500, 1500], np.int64))
    gts = [scenes.random_gt(W, H, 52 + u) for u in range(2)]
    gt = torch.from_numpy(np.stack([t[0] for t in gts])).cuda()
    mask = torch.from_numpy(np.stack([t[1] for t in gts])).cuda()
    fr = gsp.Frame(n, units, W, H, deg, deterministic=True)
    params = gsp.pack_params(g, deg)
    fr.fit_capacity(params, now)
    fr.forward(params, now, BG)
    fr.loss(gt, mask, 0.2)
    fr.blend_backward(BG)
    opt = gsp.Adam(params, deg, extent=1.0, lr_steps=100)
    p0 = params.clone()
    recs = ("xy", "conic_op", "rgb", "depth", "radius", "tiles")
    out = []
    for fused in (False, True):
        params.copy_(p0)
        opt.m.zero_()
        opt.v.zero_()
        opt.step_dev.zero_()
        fr.preprocess(params, now)
        if fused:
            opt.fused_step(fr, now, next_cams_dev=nxt)
        else:
            opt.fused_step(fr, now)
            fr.preprocess(params, nxt)
        torch.cuda.synchronize()
        assert fr.read_status() == 0
        out.append({k: getattr(fr, k)[:n].clone() for k in recs} | dict(p=params.clone(), m=opt.m.clone()))
    a, b = out
    assert torch.equal(a["p"], b["p"]) and torch.equal(a["m"], b["m"])
    assert not torch.equal(a["p"], p0)
    vis = a["radius"] > 0
    assert int(vis[:2500].sum()) > 1000 and int(vis[2500:].sum()) > 600
    for k in ("depth", "radius", "tiles"):
        assert torch.equal(a[k], b[k]), k
    for k in ("xy", "conic_op", "rgb"):
        assert torch.equal(a[k][vis], b[k][vis]), k


@pytest.mark.parametrize("sched,det", [(True, False), (False, False), (True, True)])
def test_bg_penalty_parity(sched, det):
    """Masked loss plus the background-opacity penalty (gs_bg_penalty): the loss value, dL/dT_final and every
    parameter gradient through the reverse replay (scheduled or plain kernels, float or fixed-point
    accumulation) against the oracle's penalty and its reverse replay with dL/dT_final."""
    import paper_2509_12138_gb300 as gsp
    n, deg, W, H, seed, lam, lam_bg = 1500, 2, 120, 90, 41, 0.2, 0.5
    g, cams = _case(n, deg, seed, W, H, ls=(-3.0, -1.8))
    gt, mask = scenes.random_gt(W, H, seed + 50)
    fr = gsp.Frame(n, gsp.Units.single(n), W, H, deg, deterministic=det)
    fr.use_masks = sched
    params = gsp.pack_params(g, deg)
    camd = gsp.pack_cameras(cams)
    fr.fit_capacity(params, camd)
    fr.forward(params, camd, BG)
    fr.loss(torch.from_numpy(gt).cuda(), torch.from_numpy(mask).cuda(), lam)
    dT = fr.bg_penalty(torch.from_numpy(mask).cuda(), lam_bg)
    fr.backward(params, camd, BG, dT=dT)
    torch.cuda.synchronize()
    assert fr.read_status() == 0
    cam = oracle.camera_block(cams, 0)
    g64 = gauss64(g)
    r = oracle.render(g64, cam, BG)
    lval, dimg = oracle.loss(r["img"], gt.astype(np.float64), mask, lam)
    pval, dTo = oracle.bg_penalty(r["final_T"], mask, lam_bg)
    assert pval > 0.0
    assert float(fr.loss_val.item()) == pytest.approx(lval + pval, rel=1e-4)
    assert np.allclose(dT.cpu().numpy()[0], dTo, rtol=1e-6, atol=0.0)
    g2o = oracle.render_backward(g64, cam, BG, dimg, dTo)
    go = oracle.project_backward(g64, cam, g2o)
    vis = fr.radius.cpu().numpy() > 0
    dco = fr.dco.cpu().numpy()
    for a, b in [(fr.dxy.cpu().numpy(), g2o["dxy"]), (dco[:, :3], g2o["dconic"]), (dco[:, 3], g2o["dopacity"])]:
        assert np.abs(a[vis] - b[vis]).max() <= GRAD_TOL * np.abs(b).max()
    _group_check(gsp.unpack_grads(fr.grads, deg), go, deg)
    # the penalty's share of the opacity gradient is material (the check above is not the loss alone)
    g2l = oracle.render_backward(g64, cam, BG, dimg)
    diff = np.abs(g2o["dopacity"] - g2l["dopacity"]).max()
    assert diff > 0.05 * np.abs(g2o["dopacity"]).max()
