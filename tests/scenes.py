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
