"""Small seeded scenes for the tests (built from synth; no rasterizer arithmetic)."""
import numpy as np

import synth


def front_camera(W, H, fovy_deg=60.0, eye=(0.0, 0.0, -3.0), target=(0.0, 0.0, 0.0)):
    """One camera looking from ``eye`` at ``target``."""
    cams = synth.orbital_cameras(1, 1.0, width=W, height=H, fovy_deg=fovy_deg)
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.array([0.0, 1.0, 0.0]) if abs(f[2]) > 0.99 else np.array([0.0, 0.0, 1.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    cams.viewmat[0, :, :3] = R
    cams.viewmat[0, :, 3] = -R @ eye
    cams.campos[0] = eye
    return cams


def identity_camera(W, H, fovy_deg=60.0):
    """Camera at the origin looking down +z (camera frame == world frame)."""
    cams = synth.orbital_cameras(1, 1.0, width=W, height=H, fovy_deg=fovy_deg)
    cams.viewmat[0] = np.hstack([np.eye(3), np.zeros((3, 1))]).astype(np.float32)
    cams.campos[0] = 0.0
    return cams


def random_scene(n, deg, seed, W, H, extent=1.0, log_scale_range=(-3.5, -2.0)):
    """n random Gaussians in front of a camera 3 units away."""
    g = synth.random_gaussians(n, deg, seed, extent=extent, log_scale_range=log_scale_range)
    cams = front_camera(W, H)
    return g, cams


def random_gt(W, H, seed):
    s = synth.streams(seed, ["gt", "mask"])
    gt = s["gt"].uniform(0.0, 1.0, (3, H, W)).astype(np.float32)
    mask = (s["mask"].uniform(0.0, 1.0, (H, W)) > 0.2).astype(np.uint8)
    return gt, mask


def deep_stop_scene(seed, W=32, H=32, n_faint=2100, fillers_per_tile=6300, deg=1):
    """Pixels that stop thousands of entries deep in their tile lists, for an identity camera: n_faint
    screen-filling splats of opacity 0.0045 (alpha just above 1/255 everywhere, so a pixel stops after
    ~2040 of them), interleaved in depth with small opaque fillers at each tile's corner pixel (in every
    list of their tile, blending only near that corner).  Pixels away from the corners stop after
    ~4 x 2040 list entries."""
    rng = np.random.default_rng(seed)
    cams = identity_camera(W, H)
    f, cx, cy = float(cams.fx[0]), float(cams.cx[0]), float(cams.cy[0])
    TX, TY = (W + 15) // 16, (H + 15) // 16
    z_f = rng.uniform(2.0, 4.0, n_faint)
    means = [np.stack([np.zeros(n_faint), np.zeros(n_faint), z_f], 1)]
    log_s = [np.log(100.0 * z_f / f)[:, None].repeat(3, 1)]
    logit = [np.full(n_faint, np.log(0.0045 / 0.9955))]
    for ty in range(TY):
        for tx in range(TX):
            z = rng.uniform(2.0, 4.0, fillers_per_tile)
            u, v = 16.0 * tx + 0.2, 16.0 * ty + 0.2
            means.append(np.stack([(u - cx) / f * z, (v - cy) / f * z, z], 1))
            log_s.append(np.log(0.4 * z / f)[:, None].repeat(3, 1))
            logit.append(np.full(fillers_per_tile, np.log(0.9 / 0.1)))
    n = n_faint + TX * TY * fillers_per_tile
    quats = np.zeros((n, 4))
    quats[:, 0] = 1.0
    sh = rng.normal(0.0, 0.3, (n, (deg + 1) ** 2, 3))
    g = dict(means=np.concatenate(means), log_scales=np.concatenate(log_s), quats=quats,
             logit_opacity=np.concatenate(logit), sh=sh)
    return {k: np.asarray(v, np.float32) for k, v in g.items()}, cams
