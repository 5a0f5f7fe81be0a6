"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare with the oracle under the exclusion rules for FP32-vs-FP64 near-ties."""
import math

import numpy as np
import torch

import oracle
import paper_2509_12138_gb300 as gs

TILE = 16


def gauss64(g):
    return {k: np.asarray(v, np.float64) for k, v in g.items()}


def rects(xy, radius, W, H):
    """Tile rectangles with floor((u - r)/16), floor((u + r + 15)/16), clamped.  ``xy`` is [n, 2] exact
    float64 positions, or the kernels' [n, 4] float pairs (x, y, x_lo, y_lo), whose floor is taken exactly."""
    TX, TY = (W + TILE - 1) // TILE, (H + TILE - 1) // TILE
    xy = np.asarray(xy)
    if xy.shape[1] == 4:
        hi, lo = xy[:, :2].astype(np.float64), xy[:, 2:].astype(np.float64)
        f = np.floor(hi)
        fl = (f - ((f == hi) & (lo < 0))).astype(np.int64)
        fu, fv = fl[:, 0], fl[:, 1]
    else:
        fu = np.floor(xy[:, 0]).astype(np.int64)
        fv = np.floor(xy[:, 1]).astype(np.int64)
    r = radius.astype(np.int64)
    x0 = np.clip((fu - r) // TILE, 0, TX)
    y0 = np.clip((fv - r) // TILE, 0, TY)
    x1 = np.clip((fu + r + TILE - 1) // TILE, 0, TX)
    y1 = np.clip((fv + r + TILE - 1) // TILE, 0, TY)
    out = np.stack([x0, y0, x1, y1], 1)
    out[r <= 0] = 0
    return out


def discrete_mismatch(o_proj, g_xy4, g_radius, g_tiles, W, H):
    """Gaussians whose visibility, radius, tile rectangle or tile count differ between the kernels and the
    oracle.  Returns (mismatch mask, True where every mismatch is a decision the oracle flags as a float32
    near-tie)."""
    r_gpu = rects(g_xy4, g_radius, W, H)
    vis_o, vis_g = o_proj["radius"] > 0, g_radius > 0
    mism = (vis_o != vis_g) | (g_radius != o_proj["radius"]) | np.any(r_gpu != o_proj["rect"], axis=1) \
        | (g_tiles != o_proj["tiles"])
    return mism, bool(np.all(o_proj["unstable"][mism] != 0))


def run_gpu(g, cams, deg, bg, gt=None, mask=None, lam=0.2, backward=True, units=None, max_instances=None):
    """Full pipeline on the GPU for all cameras in ``cams`` (one unit per camera unless ``units``)."""
    n = g["means"].shape[0]
    W, H = cams.width, cams.height
    units = units or gs.Units.single(n, len(cams))
    fr = gs.Frame(n, units, W, H, deg, max_instances=max_instances)
    params = gs.pack_params(g, deg)
    camd = gs.pack_cameras(cams)
    if max_instances is None:
        fr.fit_capacity(params, camd)
    fr.forward(params, camd, bg)
    out = dict(frame=fr, params=params, cams=camd)
    if gt is not None:
        gtt = torch.from_numpy(np.ascontiguousarray(gt, np.float32)).cuda()
        mk = torch.from_numpy(np.ascontiguousarray(mask, np.uint8)).cuda()
        fr.loss(gtt, mk, lam)
        out["loss"] = float(fr.loss_val.item())
        out["dimg"] = fr.dimg.cpu().numpy()
        if backward:
            fr.backward(params, camd, bg)
            out["grads"] = gs.unpack_grads(fr.grads, deg)
            out["dxy"] = fr.dxy.cpu().numpy()
            out["dco"] = fr.dco.cpu().numpy()
            out["drgb"] = fr.drgb.cpu().numpy()
    torch.cuda.synchronize()
    out["status"] = fr.read_status()
    out["img"] = fr.img.cpu().numpy()
    out["final_T"] = fr.final_T.cpu().numpy()
    out["n_contrib"] = fr.n_contrib.cpu().numpy()
    out["xy4"] = fr.xy.cpu().numpy()
    out["xy"] = fr.xy64()
    out["conic_op"] = fr.conic_op.cpu().numpy()
    out["rgb"] = fr.rgb.cpu().numpy()
    out["depth"] = fr.depth.cpu().numpy()
    out["radius"] = fr.radius.cpu().numpy()
    out["tiles"] = fr.tiles.cpu().numpy()
    out["vals"], out["ranges"] = fr.sorted_lists()
    return out


def exclusion_mask(o_proj, g_xy4, g_radius, g_tiles, margin, W, H, margin_tol=1e-5):
    """Pixels excluded from image comparison, and their causes: pixels where some blend decision of the
    oracle sits within ``margin_tol`` (relative) of its threshold, and the tiles touched by a Gaussian whose
    visibility, radius or rectangle differs between the kernels and the oracle (each such Gaussian must be
    a decision the oracle flags as a float32 near-tie).  Returns (pixels, n differing Gaussians, all flagged)."""
    TX, TY = (W + TILE - 1) // TILE, (H + TILE - 1) // TILE
    bad_tile = np.zeros((TY, TX), bool)
    mism, flagged = discrete_mismatch(o_proj, g_xy4, g_radius, g_tiles, W, H)
    r_gpu = rects(g_xy4, g_radius, W, H)
    r_orc = o_proj["rect"].astype(np.int64)
    for i in np.nonzero(mism)[0]:
        for r in (r_gpu[i], r_orc[i]):
            bad_tile[r[1]:r[3], r[0]:r[2]] = True
    pix = np.kron(bad_tile, np.ones((TILE, TILE), bool))[:H, :W]
    pix |= margin < margin_tol
    return pix, int(mism.sum()), flagged
