"""Adaptive density control on the GPU against the oracle (oracle/densify.py)."""
import math

import numpy as np
import pytest
import torch

import paper_2509_12138_gb300 as gs
from oracle import densify as D
from paper_2509_12138_gb300 import workload
from paper_2509_12138_gb300.densify import DensifyConfig, Densifier
from paper_2509_12138_gb300.train import PlainTrainer, psnr, split_views
from tests import scenes

pytestmark = pytest.mark.gpu
BG = (1.0, 1.0, 1.0)


def test_stats_parity():
    """The statistics of two steps, from seeded screen-space gradients and radii (a third of the records
    culled) written into a frame's buffers, against the oracle on the same values."""
    n, deg, W, H = 3000, 1, 120, 90
    rng = np.random.default_rng(91)
    dxy = rng.normal(0.0, 1e-4, (n, 2)).astype(np.float32)
    rad = np.where(rng.random(n) < 1 / 3, 0, rng.integers(1, 40, n)).astype(np.int32)
    fr = gs.Frame(n, gs.Units.single(n), W, H, deg)
    fr.dxy.copy_(torch.from_numpy(dxy))
    fr.radius.copy_(torch.from_numpy(rad))
    d = Densifier(n)
    d.accumulate(fr)
    d.accumulate(fr)
    torch.cuda.synchronize()
    ga, dn, mr = D.stats(np.zeros(n), np.zeros(n), np.zeros(n), dxy.astype(np.float64), rad, W, H)
    ga, dn, mr = D.stats(ga, dn, mr, dxy.astype(np.float64), rad, W, H)
    assert (rad > 0).sum() > 100
    np.testing.assert_allclose(d.grad_accum.cpu().numpy(), ga, rtol=1e-5, atol=1e-12)
    np.testing.assert_array_equal(d.denom.cpu().numpy(), dn)
    np.testing.assert_array_equal(d.max_radius.cpu().numpy(), mr)


def _random_set(n, deg, seed):
    """Gaussians and statistics whose decisions sit far from every threshold."""
    rng = np.random.default_rng(seed)
    big = rng.random(n) < 0.4
    ls = np.where(big[:, None], math.log(0.05), math.log(0.001)) + rng.uniform(-0.2, 0.2, (n, 3))
    o = np.where(rng.random(n) < 0.15, 0.001, rng.uniform(0.2, 0.9, n))
    g = {"means": rng.uniform(-1, 1, (n, 3)), "log_scales": ls, "quats": rng.normal(size=(n, 4)),
         "logit_opacity": np.log(o / (1 - o)), "sh": rng.normal(0, 0.3, (n, (deg + 1) ** 2, 3))}
    g = {k: np.asarray(v, np.float32) for k, v in g.items()}
    denom = rng.integers(0, 6, n).astype(np.float32)
    avg = np.where(rng.random(n) < 0.5, 1e-5, 1e-2).astype(np.float32)
    grad = (avg * denom).astype(np.float32)
    maxr = np.where(rng.random(n) < 0.1, 30.0, 5.0).astype(np.float32)
    return g, grad, denom, maxr


@pytest.mark.parametrize("step", [1000, 3500])
def test_plan_and_apply_parity(step):
    n, deg = 4000, 1
    g, grad, denom, maxr = _random_set(n, deg, step)
    params = gs.pack_params(g, deg)
    m = gs.pack_params({k: v + 1.0 for k, v in g.items()}, deg)
    v = gs.pack_params({k: v + 2.0 for k, v in g.items()}, deg)
    d = Densifier(n, DensifyConfig(extent=1.0))
    d.grad_accum.copy_(torch.from_numpy(grad))
    d.denom.copy_(torch.from_numpy(denom))
    d.max_radius.copy_(torch.from_numpy(maxr))
    z_np = np.random.default_rng(step + 1).standard_normal((n, 2, 3)).astype(np.float32)
    z = torch.from_numpy(z_np).cuda()
    counts = d.plan(params, step)
    po, mo, vo = d.apply(params, m, v, deg, counts, z)
    torch.cuda.synchronize()
    act = D.plan(g, grad, denom, maxr, step, extent=1.0)
    assert counts == ((act == 1).sum() + (act == 2).sum(), (act == 2).sum(), (act == 3).sum())
    assert min(counts) > 50  # every action occurs
    un = lambda t: gs.unpack_params(t, deg)
    gm = {k: np.asarray(x, np.float64) for k, x in un(m).items()}
    gv = {k: np.asarray(x, np.float64) for k, x in un(v).items()}
    ref, rm, rv = D.apply({k: np.asarray(x, np.float64) for k, x in g.items()}, gm, gv, act,
                          z_np.astype(np.float64))
    out, om, ov = un(po), un(mo), un(vo)
    n_copy = counts[0] + counts[1]
    for k in ref:
        np.testing.assert_array_equal(np.asarray(out[k][:n_copy], np.float64), ref[k][:n_copy])  # kept and copies
        np.testing.assert_array_equal(np.asarray(om[k], np.float64), rm[k])
        np.testing.assert_array_equal(np.asarray(ov[k], np.float64), rv[k])
    np.testing.assert_allclose(out["means"][n_copy:], ref["means"][n_copy:], atol=2e-6)
    np.testing.assert_allclose(out["log_scales"][n_copy:], ref["log_scales"][n_copy:], atol=2e-6)
    for k in ("quats", "logit_opacity", "sh"):
        np.testing.assert_array_equal(np.asarray(out[k][n_copy:], np.float64), ref[k][n_copy:])


def test_opacity_reset_parity():
    n, deg = 1000, 0
    g, *_ = _random_set(n, deg, 5)
    params = gs.pack_params(g, deg)
    m = gs.pack_params({k: v + 1.0 for k, v in g.items()}, deg)
    v = gs.pack_params({k: v + 2.0 for k, v in g.items()}, deg)
    m_in = {k: np.asarray(x + 1.0, np.float64) for k, x in g.items()}
    v_in = {k: np.asarray(x + 2.0, np.float64) for k, x in g.items()}
    Densifier(n).reset_opacity(params, m, v)
    rg, rm, rv = D.opacity_reset({k: np.asarray(x, np.float64) for k, x in g.items()}, m_in, v_in)
    out = gs.unpack_params(params, deg)
    np.testing.assert_allclose(out["logit_opacity"], rg["logit_opacity"], atol=1e-6)
    np.testing.assert_array_equal(gs.unpack_params(m, deg)["logit_opacity"], 0.0)
    np.testing.assert_array_equal(gs.unpack_params(m, deg)["means"], rm["means"])


def test_training_with_densification_grows_and_fits():
    scene = workload.isosurface_scene(40000, 4, 16, 128, 96, sh_degree=1, seed=7)
    train_v, test_v = split_views(16)
    sub = {k: v[::8] for k, v in scene.init.items()}  # sparse start: every 8th surface point
    sub["log_scales"] = sub["log_scales"] + math.log(2.0)
    res = {}
    for name, cfg in (("fixed", None), ("densify", DensifyConfig(start=100, stop=700, interval=100,
                                                                 reset_interval=10 ** 9, extent=1.0))):
        p = gs.pack_params(sub, 1)
        tr = PlainTrainer(p, 1, scene.cams_dev, scene.gt, scene.mask, train_v, densify=cfg, seed=1)
        for _ in range(800):
            tr.step()
        torch.cuda.synchronize()
        assert tr.check() == 0
        res[name] = (tr.params.shape[1], tr.evaluate(test_v))
    n0 = sub["means"].shape[0]
    assert res["fixed"][0] == n0 and res["densify"][0] > 1.2 * n0
    assert np.isfinite(res["densify"][1])
    assert res["densify"][1] > res["fixed"][1], res
