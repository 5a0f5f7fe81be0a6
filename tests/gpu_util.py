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
    """Tile rectangles from (x, y, radius) with floor((u - r)/16), floor((u + r + 15)/16), clamped."""
    TX, TY = (W + TILE - 1) // TILE, (H + TILE - 1) // TILE
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
    out["xy"] = fr.xy.cpu().numpy()
    out["conic_op"] = fr.conic_op.cpu().numpy()
    out["rgb"] = fr.rgb.cpu().numpy()
    out["depth"] = fr.depth.cpu().numpy()
    out["radius"] = fr.radius.cpu().numpy()
    out["tiles"] = fr.tiles.cpu().numpy()
    out["vals"], out["ranges"] = fr.sorted_lists()
    return out


def exclusion_mask(o_proj, g_xy, g_radius, tie_tiles, margin, W, H, margin_tol=1e-5):
    """Pixels excluded from image comparison: near-threshold pixels (oracle margin), and tiles touched by
    a Gaussian whose radius or rectangle differs between FP32 and FP64.  (The list order itself is decided
    on the float32 depth key on both sides, and equal keys fall back to the index, so it needs no exclusion.)"""
    TX, TY = (W + TILE - 1) // TILE, (H + TILE - 1) // TILE
    bad_tile = np.zeros((TY, TX), bool)
    r_gpu = rects(g_xy.astype(np.float64), g_radius, W, H)
    r_orc = o_proj["rect"].astype(np.int64)
    diff = np.nonzero((g_radius != o_proj["radius"]) | np.any(r_gpu != r_orc, axis=1))[0]
    for i in diff:
        for r in (r_gpu[i], r_orc[i]):
            bad_tile[r[1]:r[3], r[0]:r[2]] = True
    pix = np.kron(bad_tile, np.ones((TILE, TILE), bool))[:H, :W]
    pix |= margin < margin_tol
    return pix, len(diff)
