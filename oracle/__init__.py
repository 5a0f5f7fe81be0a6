"""FP64 CPU oracle of the Gaussian-splat rasterizer -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never calls it, and it shares no code with them.

The numerics live in plain C++ (``gs_oracle.cpp``, ``mlp_oracle.cpp``), built
with gcc into ``oracle/_build/liboracle.so`` and called through ctypes.  This
module only converts numpy arrays.  Each wrapper names the definition it
follows; the pins that check them are in ``tests/test_oracle_*.py``.

Parity status: every function here is pinned by a closed form, brute force,
a library routine, finite differences or dual numbers.  Parity unpinned: the
values of the Adam learning rates and the loss weighting (readings, not
derivable from the paper; the optimiser and the loss themselves are pinned).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = [os.path.join(_HERE, "gs_oracle.cpp"), os.path.join(_HERE, "mlp_oracle.cpp")]
_lock = threading.Lock()
_lib = None

TILE = 16


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, OpenMP).  Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SOURCES)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp] + _SOURCES
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = C.CDLL(_LIB_PATH)
            _declare(_lib)
    return _lib


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_U8 = C.POINTER(C.c_ubyte)


def _declare(L):
    L.orc_num_threads.restype = C.c_int
    L.orc_set_threads.argtypes = [C.c_int]
    L.orc_sh_basis.argtypes = [C.c_int, C.c_int, _D, _D]
    L.orc_quat_to_rot.argtypes = [C.c_int, _D, _D]
    L.orc_project.argtypes = [C.c_int, C.c_int, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _I, _D, _I, _I, _I, _D, _I]
    L.orc_bin.argtypes = [C.c_int, _D, _I, _D, C.c_int, C.c_int, C.c_longlong, _I, _I, _I, _I]
    L.orc_bin.restype = C.c_longlong
    L.orc_render.argtypes = [C.c_int, C.c_int, _D, _D, _D, _D, _D, _D, _D, _D, _D, _I, _D, _I, _D, _D]
    L.orc_render_bruteforce.argtypes = [C.c_int, C.c_int, _D, _D, _D, _D, _D, _D, _D, _D, _D, _I]
    L.orc_loss.argtypes = [_D, _D, _U8, C.c_int, C.c_int, C.c_double, _D]
    L.orc_loss.restype = C.c_double
    L.orc_loss_dir.argtypes = [_D, _D, _D, _U8, C.c_int, C.c_int, C.c_double]
    L.orc_loss_dir.restype = C.c_double
    L.orc_render_backward.argtypes = [C.c_int, C.c_int, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]
    L.orc_bg_penalty.argtypes = [_D, _U8, C.c_int, C.c_int, C.c_double, _D]
    L.orc_bg_penalty.restype = C.c_double
    L.orc_penalty_params_dir.argtypes = [C.c_int, C.c_int, _D, _D, _D, _D, _D, _D, _D, _D, _U8, C.c_double, _D]
    L.orc_penalty_params_dir.restype = C.c_double
    L.orc_project_backward.argtypes = [C.c_int, C.c_int, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]
    L.orc_loss_params_dir.argtypes = [C.c_int, C.c_int, _D, _D, _D, _D, _D, _D, _D, _D, _D, _U8,
                                      C.c_double, _D]
    L.orc_loss_params_dir.restype = C.c_double
    L.orc_adam.argtypes = [C.c_longlong, _D, _D, _D, _D, _D, C.c_double, C.c_double, C.c_double, C.c_int]
    L.orc_knn.argtypes = [C.c_int, _D, C.c_int, _I, _D]
    L.orc_owned.argtypes = [C.c_int, _D, _I, _D, _I, _U8]
    L.orc_bf16_round.argtypes = [C.c_double]
    L.orc_bf16_round.restype = C.c_double
    L.orc_mlp_features.argtypes = [C.c_int, _D, _D, _I, _D, _D]
    L.orc_mlp_forward.argtypes = [C.c_int] + [_D] * 10
    L.orc_mlp_forward_full.argtypes = [C.c_int] + [_D] * 12
    L.orc_bf16_round_array.argtypes = [C.c_longlong, _D, _D]
    L.orc_mlp_backward.argtypes = [C.c_int] + [_D] * 14
    L.orc_mlp_backward.restype = C.c_double
    L.orc_init_gaussians.argtypes = [C.c_int, _D, C.c_int, _D, C.c_double, _D, _D, _D]


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    if a is None:
        return None
    if a.dtype == np.float64:
        return a.ctypes.data_as(_D)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_I)
    if a.dtype == np.uint8:
        return a.ctypes.data_as(_U8)
    raise TypeError(a.dtype)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def n_params(deg: int) -> int:
    return 11 + 3 * (deg + 1) ** 2


def camera_block(cams, i: int) -> np.ndarray:
    """24 doubles: R[9], t[3], fx, fy, cx, cy, tan_fovx, tan_fovy, campos[3], znear, W, H."""
    vm = np.asarray(cams.viewmat[i], dtype=np.float64)
    return np.concatenate([
        vm[:, :3].reshape(-1), vm[:, 3],
        [cams.fx[i], cams.fy[i], cams.cx[i], cams.cy[i], cams.tan_fovx[i], cams.tan_fovy[i]],
        np.asarray(cams.campos[i], dtype=np.float64), [cams.znear, cams.width, cams.height],
    ]).astype(np.float64)


def _gauss(g):
    n = g["means"].shape[0]
    sh = _d(g["sh"]).reshape(n, -1)
    deg = int(round(np.sqrt(sh.shape[1] // 3))) - 1
    return n, deg, _d(g["means"]), _d(g["log_scales"]), _d(g["quats"]), _d(g["logit_opacity"]), sh


def flatten_params(g) -> np.ndarray:
    """[n, n_params] in the order mean(3), log-scale(3), quat(4), logit(1), SH (coeff-major)."""
    n, deg, m, ls, q, lo, sh = _gauss(g)
    return np.concatenate([m, ls, q, lo[:, None], sh], axis=1)


def unflatten_params(v: np.ndarray, deg: int):
    v = np.asarray(v)
    n = v.shape[0]
    return dict(means=v[:, 0:3], log_scales=v[:, 3:6], quats=v[:, 6:10], logit_opacity=v[:, 10],
                sh=v[:, 11:].reshape(n, (deg + 1) ** 2, 3))


def sh_basis(dirs, deg: int) -> np.ndarray:
    dirs = _d(dirs)
    n = dirs.shape[0]
    out = np.zeros((n, (deg + 1) ** 2))
    lib().orc_sh_basis(n, deg, _p(dirs), _p(out))
    return out


def quat_to_rot(q) -> np.ndarray:
    q = _d(q).reshape(-1, 4)
    R = np.zeros((q.shape[0], 9))
    lib().orc_quat_to_rot(q.shape[0], _p(q), _p(R))
    return R.reshape(-1, 3, 3)


def project(g, cam):
    n, deg, m, ls, q, lo, sh = _gauss(g)
    cam = _d(cam)
    out = dict(xy=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)),
               clamp=np.zeros(n, np.int32), depth=np.zeros(n), radius=np.zeros(n, np.int32),
               rect=np.zeros((n, 4), np.int32), tiles=np.zeros(n, np.int32), cov2d=np.zeros((n, 3)),
               unstable=np.zeros(n, np.int32))
    lib().orc_project(n, deg, _p(m), _p(ls), _p(q), _p(lo), _p(sh), _p(cam), _p(out["xy"]), _p(out["conic"]),
                      _p(out["opacity"]), _p(out["rgb"]), _p(out["clamp"]), _p(out["depth"]),
                      _p(out["radius"]), _p(out["rect"]), _p(out["tiles"]), _p(out["cov2d"]), _p(out["unstable"]))
    # depth: the float32 rounding of the FP64 camera-space z (the sort key); unstable: bits 1 (near
    # cull), 2 (radius), 4 (tile rectangle) of the decisions a float32 evaluation may take the other
    # way, by the error model stated in gs_oracle.cpp
    return out


def bin_sort(xy, radius, depth, W: int, H: int):
    """Instances ordered by (tile, depth, index) and per-tile [start, end)."""
    xy, radius, depth = _d(xy), _i(radius), _d(depth)
    n = xy.shape[0]
    TX, TY = (W + TILE - 1) // TILE, (H + TILE - 1) // TILE
    ranges = np.zeros((TX * TY, 2), np.int32)
    ties = np.zeros(TX * TY, np.int32)
    dummy = np.zeros(1, np.int32)
    I = lib().orc_bin(n, _p(xy), _p(radius), _p(depth), W, H, 0, _p(dummy), _p(dummy), _p(ranges), _p(ties))
    idx = np.zeros(max(I, 1), np.int32)
    tile = np.zeros(max(I, 1), np.int32)
    lib().orc_bin(n, _p(xy), _p(radius), _p(depth), W, H, I, _p(idx), _p(tile), _p(ranges), _p(ties))
    return dict(idx=idx[:I], tile=tile[:I], ranges=ranges, tie_tiles=ties)


def render(g, cam, bg):
    n, deg, m, ls, q, lo, sh = _gauss(g)
    cam, bg = _d(cam), _d(bg)
    W, H = int(cam[22]), int(cam[23])
    TX, TY = (W + TILE - 1) // TILE, (H + TILE - 1) // TILE
    img = np.zeros((3, H, W))
    T = np.zeros((H, W))
    nc = np.zeros((H, W), np.int32)
    margin = np.zeros((H, W))
    ties = np.zeros(TX * TY, np.int32)
    stop_margin = np.zeros((H, W))
    t_err = np.zeros((H, W))
    lib().orc_render(n, deg, _p(m), _p(ls), _p(q), _p(lo), _p(sh), _p(cam), _p(bg), _p(img), _p(T), _p(nc),
                     _p(margin), _p(ties), _p(stop_margin), _p(t_err))
    # stop_margin / t_err: the early-stop decision's own relative distance to T_MIN and a bound on the
    # relative float32 error of T at that point (see blend_pixel)
    return dict(img=img, final_T=T, n_contrib=nc, margin=margin, tie_tiles=ties, stop_margin=stop_margin,
                t_err=t_err)


def render_bruteforce(g, cam, bg):
    n, deg, m, ls, q, lo, sh = _gauss(g)
    cam, bg = _d(cam), _d(bg)
    W, H = int(cam[22]), int(cam[23])
    img = np.zeros((3, H, W))
    T = np.zeros((H, W))
    nc = np.zeros((H, W), np.int32)
    lib().orc_render_bruteforce(n, deg, _p(m), _p(ls), _p(q), _p(lo), _p(sh), _p(cam), _p(bg), _p(img),
                                _p(T), _p(nc))
    return dict(img=img, final_T=T, n_contrib=nc)


def loss(img, gt, mask, lam: float, grad: bool = True):
    img, gt = _d(img), _d(gt)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    H, W = mask.shape
    d = np.zeros_like(img) if grad else None
    val = lib().orc_loss(_p(img), _p(gt), _p(mask), W, H, float(lam), _p(d) if grad else None)
    return (val, d) if grad else val


def loss_dir(img, direction, gt, mask, lam: float) -> float:
    img, direction, gt = _d(img), _d(direction), _d(gt)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    H, W = mask.shape
    return lib().orc_loss_dir(_p(img), _p(direction), _p(gt), _p(mask), W, H, float(lam))


def render_backward(g, cam, bg, dimg, dT=None):
    """Screen-space gradients from dL/dimage and, optionally, dL/dT_final ([H, W]) of a loss term on the
    pixels' final transmittance (the background-opacity penalty)."""
    n, deg, m, ls, q, lo, sh = _gauss(g)
    cam, bg, dimg = _d(cam), _d(bg), _d(dimg)
    dT = None if dT is None else _d(dT)
    out = dict(dxy=np.zeros((n, 2)), dconic=np.zeros((n, 3)), dopacity=np.zeros(n), drgb=np.zeros((n, 3)))
    lib().orc_render_backward(n, deg, _p(m), _p(ls), _p(q), _p(lo), _p(sh), _p(cam), _p(bg), _p(dimg),
                              _p(dT) if dT is not None else None,
                              _p(out["dxy"]), _p(out["dconic"]), _p(out["dopacity"]), _p(out["drgb"]))
    return out


def bg_penalty(final_T, mask, lam: float):
    """Background-opacity penalty of one view: lam x mean of (1 - T_final) over the pixels outside the mask
    (0 if there are none), and its gradient dpenalty/dT_final [H, W]."""
    final_T = _d(final_T)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    H, W = mask.shape
    dT = np.zeros((H, W))
    val = lib().orc_bg_penalty(_p(final_T), _p(mask), W, H, float(lam), _p(dT))
    return val, dT


def penalty_params_dir(g, tangent, cam, bg, mask, lam: float):
    """(penalty, exact directional derivative along ``tangent`` [n, n_params]) by dual numbers."""
    n, deg, m, ls, q, lo, sh = _gauss(g)
    tangent, cam, bg = _d(tangent), _d(cam), _d(bg)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    dp = np.zeros(1)
    v = lib().orc_penalty_params_dir(n, deg, _p(m), _p(ls), _p(q), _p(lo), _p(sh), _p(tangent), _p(cam), _p(bg),
                                     _p(mask), float(lam), _p(dp))
    return v, float(dp[0])


def project_backward(g, cam, g2d):
    n, deg, m, ls, q, lo, sh = _gauss(g)
    cam = _d(cam)
    grads = np.zeros((n, n_params(deg)))
    lib().orc_project_backward(n, deg, _p(m), _p(ls), _p(q), _p(lo), _p(sh), _p(cam), _p(_d(g2d["dxy"])),
                               _p(_d(g2d["dconic"])), _p(_d(g2d["dopacity"])), _p(_d(g2d["drgb"])), _p(grads))
    return grads


def loss_params_dir(g, tangent, cam, bg, gt, mask, lam: float):
    """(loss, exact directional derivative along ``tangent`` [n, n_params])."""
    n, deg, m, ls, q, lo, sh = _gauss(g)
    tangent, cam, bg, gt = _d(tangent), _d(cam), _d(bg), _d(gt)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    dl = np.zeros(1)
    v = lib().orc_loss_params_dir(n, deg, _p(m), _p(ls), _p(q), _p(lo), _p(sh), _p(tangent), _p(cam), _p(bg),
                                  _p(gt), _p(mask), float(lam), _p(dl))
    return v, float(dl[0])


def loss_and_grads(g, cam, bg, gt, mask, lam: float):
    """Loss of one view and its gradient w.r.t. all parameters ([n, n_params]).

    Reverse replay of the blend for the screen-space gradients, then the
    dual-number Jacobian of the projection.
    """
    r = render(g, cam, bg)
    val, dimg = loss(r["img"], gt, mask, lam, grad=True)
    g2d = render_backward(g, cam, bg, dimg)
    grads = project_backward(g, cam, g2d)
    return dict(loss=val, grads=grads, render=r, dimg=dimg, g2d=g2d)


def adam(p, g, m, v, lr, beta1: float, beta2: float, eps: float, step: int):
    p, m, v = _d(p).copy(), _d(m).copy(), _d(v).copy()
    g = _d(g)
    lr = _d(np.broadcast_to(lr, p.shape))
    lib().orc_adam(p.size, _p(p), _p(g), _p(m), _p(v), _p(lr), beta1, beta2, eps, int(step))
    return p, m, v


def knn(pts, k: int):
    pts = _d(pts)
    n = pts.shape[0]
    idx = np.zeros((n, k), np.int32)
    dist = np.zeros((n, k))
    lib().orc_knn(n, _p(pts), k, _p(idx), _p(dist))
    return idx, dist


def owned(means, part_of, boxes, closed_hi):
    means, boxes = _d(means), _d(boxes)
    part_of, closed_hi = _i(part_of), _i(closed_hi)
    keep = np.zeros(means.shape[0], np.uint8)
    lib().orc_owned(means.shape[0], _p(means), _p(part_of), _p(boxes), _p(closed_hi), _p(keep))
    return keep.astype(bool)


def bf16_round(x):
    """Nearest bfloat16 value (ties to even) of every element, as float64."""
    a = _d(x)
    out = np.zeros_like(a)
    lib().orc_bf16_round_array(a.size, _p(a), _p(out))
    return out


def mlp_features(pts, nrm, knn_idx, knn_dist):
    pts, nrm, knn_dist = _d(pts), _d(nrm), _d(knn_dist)
    knn_idx = _i(knn_idx)
    n = pts.shape[0]
    X = np.zeros((n, 112))
    lib().orc_mlp_features(n, _p(pts), _p(nrm), _p(knn_idx), _p(knn_dist), _p(X))
    return X


def mlp_forward(X, w):
    X = _d(X)
    n = X.shape[0]
    H1, H2, Y = np.zeros((n, 64)), np.zeros((n, 64)), np.zeros((n, 8))
    ws = [_d(w[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
    A1, A2 = np.zeros((n, 64)), np.zeros((n, 64))
    lib().orc_mlp_forward_full(n, _p(X), *[_p(a) for a in ws], _p(H1), _p(H2), _p(Y), _p(A1), _p(A2))
    # H1, H2: post-ReLU activations before their bf16 rounding; A1, A2: the pre-activations
    return dict(H1=H1, H2=H2, Y=Y, A1=A1, A2=A2)


def mlp_backward(X, w, T):
    X, T = _d(X), _d(T)
    n = X.shape[0]
    ws = [_d(w[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
    g = dict(W1=np.zeros((112, 64)), b1=np.zeros(64), W2=np.zeros((64, 64)), b2=np.zeros(64),
             W3=np.zeros((64, 8)), b3=np.zeros(8))
    L = lib().orc_mlp_backward(n, _p(X), *[_p(a) for a in ws], _p(T),
                               *[_p(g[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
    return L, g


def init_gaussians(knn_dist, Y=None, logit_default=math.log(0.1 / 0.9)):
    """(log_scales [n,3], quats [n,4], logit [n]) of the plain (Y None) or learned initialiser."""
    knn_dist = _d(knn_dist)
    n, k = knn_dist.shape
    ls, q, lo = np.zeros((n, 3)), np.zeros((n, 4)), np.zeros(n)
    Yd = _d(Y) if Y is not None else None
    lib().orc_init_gaussians(n, _p(knn_dist), k, _p(Yd), float(logit_default), _p(ls), _p(q), _p(lo))
    return ls, q, lo
