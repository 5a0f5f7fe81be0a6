"""Parity at the benchmark's full size, in the launch configuration the benchmark times.

10M Gaussians (SH3, 16-mode interface), 1920x1080, the benchmark's Frame (instance capacity 6N, blend
schedule with 1024-entry chunks, chunk-parallel forward) after a few training steps.  The oracle cannot
render the whole view, so it renders tile-aligned 64x64 windows (same intrinsics, principal point shifted by
the window's origin) from the Gaussians that reach them: among them the window holding the view's longest
tile list.  Compared there: the tile lists (bit-exact, oracle binning fed the GPU's float32 projections),
pixel values, final T and n_contrib (outside near-threshold pixels), and the screen-space gradients of every
Gaussian whose tile rectangle lies inside the window (all of its pixels are in the window)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2509_12138_gb300 as gs
from paper_2509_12138_gb300 import workload
from tests.gpu_util import exclusion_mask, gauss64, rects

pytestmark = pytest.mark.gpu
N, W, H, WIN = 10_000_000, 1920, 1080, 64
IMG_TOL, GRAD_TOL = 1e-4, 1e-3
# Walks of tens of thousands of entries over thin splats: float32 conics of ill-conditioned 2D covariances
# carry up to ~3e-4 relative error (an alpha 1.4e-4 from 1/255 was seen decided the other way), so decisions
# within 3e-4 of a threshold are not compared (1e-5 in the small tests), and neither are early stops within
# four times the float32 error bound of T (oracle t_err).
MARGIN_TOL = 3e-4


@pytest.fixture(scope="module")
def full():
    scene = workload.isosurface_scene(N, 16, 8, W, H, sh_degree=3, seed=0)
    params = gs.pack_params(scene.init, 3)
    frame = gs.Frame(N, gs.Units.single(N), W, H, 3, max_instances=6 * N)
    opt = gs.Adam(params, 3, extent=1.0, lr_steps=7000)
    bg = scene.bg
    for v in range(3):  # a few optimiser steps, as the benchmark's warm-up
        cam = scene.cam(v)
        frame.preprocess(params, cam)
        frame.sort()
        frame.render(bg)
        frame.loss(scene.gt[v:v + 1], scene.mask[v:v + 1], 0.2)
        frame.blend_backward(bg)
        opt.fused_step(frame, cam)
    v = 5
    cam = scene.cam(v)
    frame.preprocess(params, cam)
    frame.sort()
    frame.render(bg)
    frame.loss(scene.gt[v:v + 1], scene.mask[v:v + 1], 0.2)
    frame.blend_backward(bg)
    torch.cuda.synchronize()
    assert frame.read_status() == 0
    vals, ranges = frame.sorted_lists()
    out = dict(img=frame.img[0].cpu().numpy(), final_T=frame.final_T[0].cpu().numpy(),
               n_contrib=frame.n_contrib[0].cpu().numpy(), dimg=frame.dimg[0].cpu().numpy(),
               xy=frame.xy.cpu().numpy(), radius=frame.radius.cpu().numpy(), depth=frame.depth.cpu().numpy(),
               dxy=frame.dxy.cpu().numpy(), dco=frame.dco.cpu().numpy(), drgb=frame.drgb.cpu().numpy(),
               vals=vals, ranges=ranges, g=gauss64(gs.unpack_params(params, 3)),
               cam=oracle.camera_block(scene.cams, v), bg=np.asarray(bg, np.float64))
    del frame, opt, params, scene
    torch.cuda.empty_cache()
    return out


def _windows(full):
    TX = (W + 15) // 16
    L = full["ranges"][:, 1] - full["ranges"][:, 0]
    heavy = int(np.argmax(L))
    rng = np.random.default_rng(0)
    covered = np.nonzero(L > 0)[0]
    picks = [heavy] + [int(t) for t in rng.choice(covered, 2, replace=False)]
    out = []
    for t in picks:
        tx, ty = t % TX, t // TX
        x0 = min(max(tx - 1, 0), (W - WIN) // 16) * 16
        y0 = min(max(ty - 1, 0), (H - WIN) // 16) * 16
        out.append((x0, y0))
    return out, int(L.max())


def _exclusion(op, xy_w, rad_gpu, margin):
    """Pixels not compared: near-threshold pixels (oracle margin), and, for each Gaussian whose float32 tile
    rectangle differs from the FP64 one, the pixels of the tiles in which only one side lists it where its
    alpha could reach 1/255 (half of it, for slack).  Lists with tens of thousands of entries always hold some
    such Gaussian, so excluding whole tiles would exclude most of a heavy window."""
    bad = margin < MARGIN_TOL
    r_gpu = rects(xy_w.astype(np.float64), rad_gpu, WIN, WIN)
    r_orc = op["rect"].astype(np.int64)
    yy, xx = np.mgrid[0:WIN, 0:WIN].astype(np.float64)
    for i in np.nonzero(np.any(r_gpu != r_orc, axis=1))[0]:
        only = np.zeros((WIN // 16, WIN // 16), bool)
        for r, s in ((r_gpu[i], 1), (r_orc[i], -1)):
            m = np.zeros_like(only)
            m[r[1]:r[3], r[0]:r[2]] = True
            only ^= m
        if not only.any():
            continue
        a, b, c = op["conic"][i]
        dx, dy = op["xy"][i][0] - xx, op["xy"][i][1] - yy
        alpha = op["opacity"][i] * np.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy)
        bad |= np.kron(only, np.ones((16, 16), bool)) & (alpha >= 0.5 / 255.0)
    return bad


def _window_cam(cam, x0, y0):
    c = cam.copy()
    c[14] -= x0
    c[15] -= y0
    c[22], c[23] = WIN, WIN
    return c


@pytest.mark.parametrize("k", [0, 1, 2])
def test_window_parity(full, k):
    wins, longest = _windows(full)
    assert longest > 20000  # the view's heaviest list is in window 0
    x0, y0 = wins[k]
    cw = _window_cam(full["cam"], x0, y0)
    g = full["g"]
    # Gaussians that reach the window by the oracle's FP64 projection or by the GPU's float32 one
    TW = WIN // 16
    r_full = rects(full["xy"].astype(np.float64), full["radius"], W, H)
    gpu_reach = ((full["radius"] > 0) & (r_full[:, 0] < x0 // 16 + TW) & (r_full[:, 2] > x0 // 16)
                 & (r_full[:, 1] < y0 // 16 + TW) & (r_full[:, 3] > y0 // 16))
    sel = np.nonzero(gpu_reach | (oracle.project(g, cw)["tiles"] > 0))[0]
    sub = {key: val[sel] for key, val in g.items()}
    # lists: the oracle's binning of the GPU's own float32 projections equals the GPU's lists for the window
    xy_w = full["xy"][sel].astype(np.float64) - np.array([x0, y0], np.float64)
    L = oracle.bin_sort(xy_w, full["radius"][sel], full["depth"][sel].astype(np.float64), WIN, WIN)
    TX = (W + 15) // 16
    for wy in range(TW):
        for wx in range(TW):
            t = (y0 // 16 + wy) * TX + (x0 // 16 + wx)
            a, b = full["ranges"][t]
            oa, ob = L["ranges"][wy * TW + wx]
            assert np.array_equal(full["vals"][a:b], sel[L["idx"][oa:ob]])
    # image, final T, n_contrib
    o = oracle.render(sub, cw, full["bg"])
    op = oracle.project(sub, cw)
    stop = o["stop_margin"] < 4.0 * o["t_err"]
    excl = _exclusion(op, xy_w, full["radius"][sel], o["margin"]) | stop
    assert excl.mean() < 0.15, excl.mean()
    # float32 compositing over thousands of entries: |dT| <= t_err T and |dC| <= t_err (oracle's bound on
    # the relative float32 error of T), so a pixel may differ by 2 t_err on top of the small tests' 1e-4
    img = full["img"][:, y0:y0 + WIN, x0:x0 + WIN]
    tol = IMG_TOL + 2.0 * o["t_err"]
    assert np.all((np.abs(img - o["img"]).max(axis=0) <= tol)[~excl])
    dT = np.abs(full["final_T"][y0:y0 + WIN, x0:x0 + WIN] - o["final_T"])
    over = (dT > IMG_TOL + o["t_err"] * o["final_T"]) & ~excl
    if over.any():
        y, x = np.argwhere(over)[0]
        pytest.fail(f"final_T at ({y},{x}): gpu {full['final_T'][y0 + y, x0 + x]} oracle {o['final_T'][y, x]} "
                    f"t_err {o['t_err'][y, x]} margin {o['margin'][y, x]} stop_margin {o['stop_margin'][y, x]} "
                    f"n_contrib gpu {full['n_contrib'][y0 + y, x0 + x]} oracle {o['n_contrib'][y, x]} "
                    f"pixels over {int(over.sum())}")
    # n_contrib is a position in the tile's list: compare it in the tiles whose lists agree entry for entry
    # (no Gaussian with a different float32 / FP64 rectangle), outside near-threshold pixels
    tile_excl, _ = exclusion_mask(op, xy_w.astype(np.float32), full["radius"][sel], o["tie_tiles"], o["margin"],
                                  WIN, WIN, margin_tol=MARGIN_TOL)
    tile_excl |= stop
    assert tile_excl.mean() < 0.5
    assert np.array_equal(full["n_contrib"][y0:y0 + WIN, x0:x0 + WIN][~tile_excl], o["n_contrib"][~tile_excl])
    # screen-space gradients of the Gaussians whose whole rectangle lies in the window
    d = oracle.render_backward(sub, cw, full["bg"], full["dimg"][:, y0:y0 + WIN, x0:x0 + WIN].astype(np.float64))
    r = rects(full["xy"][sel].astype(np.float64), full["radius"][sel], W, H)
    inside = ((r[:, 0] >= x0 // 16) & (r[:, 2] <= x0 // 16 + TW) & (r[:, 1] >= y0 // 16) & (r[:, 3] <= y0 // 16 + TW)
              & (full["radius"][sel] > 0))
    # ... whose footprint (alpha >= 1/255, with slack) holds no excluded pixel: only those pixels add to
    # a Gaussian's gradient
    touches_excl = np.zeros(len(sel), bool)
    yy, xx = np.mgrid[0:WIN, 0:WIN].astype(np.float64)
    for i in np.nonzero(inside)[0]:
        a, b, c = op["conic"][i]
        dx, dy = op["xy"][i][0] - xx, op["xy"][i][1] - yy
        foot = op["opacity"][i] * np.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy) >= 0.5 / 255.0
        touches_excl[i] = (foot & excl).any()
    use = inside & ~touches_excl
    assert use.sum() > 100, (inside.sum(), use.sum())
    gpu = {"dxy": full["dxy"][sel][use], "dconic": full["dco"][sel][use][:, :3],
           "dopacity": full["dco"][sel][use][:, 3], "drgb": full["drgb"][sel][use][:, :3]}
    # The chunked reverse replay starts each chunk from the forward's checkpoint (T and the colour behind the
    # boundary, composited back to front from the chunks' partials); float32 T recovered by division along
    # chunks of up to 1024 entries keeps 99.9% of the values within the small tests' 1e-3 of the group's scale
    # and all within 2e-3.
    for key in gpu:
        ref = d[key][use]
        sc = np.abs(ref).max()
        err = np.abs(gpu[key] - ref) / sc
        assert sc > 0 and np.quantile(err, 0.999) <= GRAD_TOL and err.max() <= 2 * GRAD_TOL, (key, err.max())
