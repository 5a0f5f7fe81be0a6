"""Pins of the oracle's binning, sort and blend.

* single Gaussian: closed-form pixel colour;
* brute force: every pixel independently collects, depth-sorts and blends
  its candidates; the tile path must agree exactly (same FP64 arithmetic);
* invariants of lists and transmittance; opacity -> 0 gives the background;
  an opaque front splat hides what is behind it.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import scenes

BG_W = np.ones(3)


def _iso(means, sig, logit, rgb):
    n = len(means)
    y00 = 0.5 / math.sqrt(math.pi)
    sh = np.zeros((n, 1, 3))
    sh[:, 0, :] = (np.asarray(rgb, np.float64) - 0.5) / y00
    return dict(means=np.asarray(means, np.float64), log_scales=np.full((n, 3), math.log(sig)),
                quats=np.tile([1.0, 0, 0, 0], (n, 1)), logit_opacity=np.full(n, float(logit)), sh=sh)


def test_single_gaussian_closed_form():
    """C(p) = a(p) c + (1 - a(p)) bg with a = min(0.99, o exp(-d^2 / (2 s2))), s2 = (f sigma/z)^2 + 0.3,
    cut below 1/255 and outside the tile rectangle."""
    W, H = 80, 64
    cams = scenes.identity_camera(W, H)
    cam = oracle.camera_block(cams, 0)
    f, cx, cy = float(cams.fx[0]), float(cams.cx[0]), float(cams.cy[0])
    bg = np.array([0.2, 0.7, 1.0])
    for z, sig, logit in [(2.0, 0.02, 2.0), (3.0, 0.05, 0.0), (1.5, 0.004, 6.0)]:
        g = _iso([[0.0, 0.0, z]], sig, logit, [[0.9, 0.3, 0.1]])
        r = oracle.render(g, cam, bg)
        s2 = (f * sig / z) ** 2 + 0.3
        o = 1 / (1 + math.exp(-logit))
        rad = math.ceil(3 * math.sqrt(s2 + math.sqrt(0.1)))
        x0, x1 = math.floor((math.floor(cx) - rad) / 16), math.floor((math.floor(cx) + rad + 15) / 16)
        y0, y1 = math.floor((math.floor(cy) - rad) / 16), math.floor((math.floor(cy) + rad + 15) / 16)
        py, px = np.mgrid[0:H, 0:W]
        d2 = (px - cx) ** 2 + (py - cy) ** 2
        a = np.minimum(0.99, o * np.exp(-0.5 * d2 / s2))
        inrect = (px // 16 >= x0) & (px // 16 < x1) & (py // 16 >= y0) & (py // 16 < y1)
        a = np.where((a >= 1 / 255) & inrect, a, 0.0)
        col = np.array([0.9, 0.3, 0.1])
        expect = a[None] * col[:, None, None] + (1 - a[None]) * bg[:, None, None]
        assert np.abs(r["img"] - expect).max() < 1e-12
        assert np.abs(r["final_T"] - (1 - a)).max() < 1e-12


def test_two_gaussians_front_to_back_closed_form():
    """Two coincident splats: C = a1 c1 + (1-a1) a2 c2 + (1-a1)(1-a2) bg, nearer one first."""
    W, H = 32, 32
    cams = scenes.identity_camera(W, H)
    cam = oracle.camera_block(cams, 0)
    # identical screen footprint: same sigma/z ratio
    g = _iso([[0, 0, 2.0], [0, 0, 1.0]], 0.02, 0.0, [[1, 0, 0], [0, 1, 0]])
    g["log_scales"][1] = math.log(0.01)
    r = oracle.render(g, cam, BG_W)
    cx = float(cams.cx[0])
    p = (int(cx), int(cx))
    f = float(cams.fx[0])
    s2 = (f * 0.01) ** 2 + 0.3
    d2 = (p[0] - cx) ** 2 + (p[1] - cx) ** 2
    a = 0.5 * math.exp(-0.5 * d2 / s2)
    expect = a * np.array([0, 1, 0]) + (1 - a) * a * np.array([1, 0, 0]) + (1 - a) ** 2 * BG_W
    assert np.allclose(r["img"][:, p[1], p[0]], expect, atol=1e-12)


@pytest.mark.parametrize("n,W,H,seed", [(40, 64, 64, 0), (64, 48, 40, 1), (500, 100, 80, 2), (300, 33, 17, 3)])
def test_tile_path_equals_bruteforce(n, W, H, seed):
    g, cams = scenes.random_scene(n, 3, seed, W, H, extent=0.8, log_scale_range=(-3.0, -1.5))
    cam = oracle.camera_block(cams, 0)
    bg = np.array([0.1, 0.5, 0.9])
    a = oracle.render(g, cam, bg)
    b = oracle.render_bruteforce(g, cam, bg)
    assert np.array_equal(a["img"], b["img"])
    assert np.array_equal(a["final_T"], b["final_T"])
    assert np.array_equal(a["n_contrib"], b["n_contrib"])


def test_list_invariants():
    g, cams = scenes.random_scene(800, 1, 7, 120, 90, extent=0.9)
    cam = oracle.camera_block(cams, 0)
    p = oracle.project(g, cam)
    L = oracle.bin_sort(p["xy"], p["radius"], p["depth"], 120, 90)
    assert len(L["idx"]) == int(p["tiles"].sum())
    rng = L["ranges"]
    assert (rng[:, 1] - rng[:, 0]).sum() == len(L["idx"])
    for t in range(rng.shape[0]):
        s, e = rng[t]
        assert np.all(L["tile"][s:e] == t)
        d = p["depth"][L["idx"][s:e]]
        assert np.all(np.diff(d) >= 0)
        # ties broken by index
        same = np.diff(d) == 0
        assert np.all(np.diff(L["idx"][s:e])[same] > 0)
        # each listed Gaussian's rectangle contains the tile
        tx, ty = t % 8, t // 8
        r = p["rect"][L["idx"][s:e]]
        assert np.all((r[:, 0] <= tx) & (tx < r[:, 2]) & (r[:, 1] <= ty) & (ty < r[:, 3]))


def test_transmittance_and_background_invariants():
    g, cams = scenes.random_scene(600, 0, 8, 96, 64)
    cam = oracle.camera_block(cams, 0)
    bg = np.array([0.3, 0.6, 0.9])
    r = oracle.render(g, cam, bg)
    assert r["final_T"].min() >= 1e-4 and r["final_T"].max() <= 1.0
    # opacity -> 0: every alpha falls below 1/255 and the image is the background
    g0 = dict(g)
    g0["logit_opacity"] = np.full_like(g["logit_opacity"], -30.0)
    r0 = oracle.render(g0, cam, bg)
    assert np.array_equal(r0["img"], np.broadcast_to(bg[:, None, None], r0["img"].shape))
    assert np.all(r0["final_T"] == 1.0) and np.all(r0["n_contrib"] == 0)


def test_opaque_front_gaussian_hides_background():
    """A large, fully opaque splat in front: alpha = 0.99 at its centre, so C = 0.99 c + 0.01 (behind)."""
    W, H = 48, 48
    cams = scenes.identity_camera(W, H)
    cam = oracle.camera_block(cams, 0)
    g = _iso([[0, 0, 1.0], [0.05, 0.0, 3.0]], 0.2, 20.0, [[0.2, 0.4, 0.6], [1.0, 0.0, 0.0]])
    r = oracle.render(g, cam, np.zeros(3))
    c = r["img"][:, 24, 24]
    assert np.all(np.abs(c - 0.99 * np.array([0.2, 0.4, 0.6])) <= 0.01 * 1.0 + 1e-12)


def test_early_stop_semantics():
    """Stacked opaque splats: each takes T down by (1 - 0.99); the entry that would bring T below 1e-4
    is not blended, so exactly two contribute and final T = 1e-4 (0.01^2)."""
    W, H = 33, 33  # principal point (16, 16) is a pixel centre
    cams = scenes.identity_camera(W, H)
    cam = oracle.camera_block(cams, 0)
    zs = [1.0, 1.1, 1.2, 1.3]
    g = _iso([[0, 0, z] for z in zs], 0.3, 30.0, [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]])
    r = oracle.render(g, cam, np.zeros(3))
    c = int(cams.cx[0])
    assert r["n_contrib"][c, c] == 2
    assert abs(r["final_T"][c, c] - 1e-4) < 1e-15
    expect = 0.99 * np.array([1, 0, 0]) + 0.01 * 0.99 * np.array([0, 1, 0])
    assert np.allclose(r["img"][:, c, c], expect, atol=1e-12)


def test_bin_sort_matches_numpy_lexsort():
    """Binning + sort equals a numpy lexsort over (tile, depth, index) of the duplicated instances."""
    g, cams = scenes.random_scene(400, 0, 9, 130, 70, extent=1.0)
    cam = oracle.camera_block(cams, 0)
    p = oracle.project(g, cam)
    L = oracle.bin_sort(p["xy"], p["radius"], p["depth"], 130, 70)
    TX = 9
    tiles, depth, idx = [], [], []
    for i in range(400):
        if p["radius"][i] == 0:
            continue
        x0, y0, x1, y1 = p["rect"][i]
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                tiles.append(ty * TX + tx)
                depth.append(p["depth"][i])
                idx.append(i)
    order = np.lexsort((np.array(idx), np.array(depth), np.array(tiles)))
    assert np.array_equal(np.array(idx)[order], L["idx"])
    assert np.array_equal(np.array(tiles)[order], L["tile"])
