"""Pins of the oracle's geometry: SH basis, quaternion rotation, EWA projection, tile rectangles.

Each check compares the oracle with something other than itself: a library
routine (scipy), an independent formula (Hamilton product, numerical
Jacobian), a closed form, or a quadrature identity.
"""
import math

import numpy as np
import pytest
import scipy.special as sps

import oracle
from tests import scenes


def _quadrature(nz=24, nphi=48):
    z, wz = np.polynomial.legendre.leggauss(nz)
    phi = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    Z, P = np.meshgrid(z, phi, indexing="ij")
    W = np.outer(wz, np.full(nphi, 2 * math.pi / nphi))
    s = np.sqrt(1 - Z ** 2)
    dirs = np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3)
    return dirs, W.reshape(-1)


def test_sh_orthonormal():
    """Gram matrix of the 16 real SH functions on the sphere is the identity."""
    dirs, w = _quadrature()
    Y = oracle.sh_basis(dirs, 3)
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_matches_scipy_convention():
    """Real SH (Condon-Shortley phase, m = -l..l) equals sqrt(2) Re / Im of scipy's complex Y_l^m."""
    rng = np.random.default_rng(1)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = oracle.sh_basis(d, 3)
    for l in range(4):
        for m in range(-l, l + 1):
            c = sps.sph_harm_y(l, abs(m), theta, phi)
            if m == 0:
                ref = c.real
            elif m > 0:
                ref = math.sqrt(2) * c.real
            else:
                ref = math.sqrt(2) * c.imag
            assert np.abs(Y[:, l * l + l + m] - ref).max() < 1e-12, (l, m)


def test_sh_degree1_closed_form():
    """Degree-1 functions are -sqrt(3/4pi) y, sqrt(3/4pi) z, -sqrt(3/4pi) x."""
    rng = np.random.default_rng(2)
    d = rng.standard_normal((50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle.sh_basis(d, 1)
    c = math.sqrt(3 / (4 * math.pi))
    assert np.allclose(Y[:, 0], 0.5 / math.sqrt(math.pi), atol=1e-15)
    assert np.allclose(Y[:, 1], -c * d[:, 1], atol=1e-14)
    assert np.allclose(Y[:, 2], c * d[:, 2], atol=1e-14)
    assert np.allclose(Y[:, 3], -c * d[:, 0], atol=1e-14)


def _hamilton(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def test_quaternion_rotation():
    """R(q) is orthonormal with det 1 and equals the sandwich q v q* (unnormalised q allowed)."""
    rng = np.random.default_rng(3)
    q = rng.standard_normal((100, 4)) * rng.uniform(0.3, 3.0, (100, 1))
    R = oracle.quat_to_rot(q)
    for i in range(100):
        assert np.abs(R[i] @ R[i].T - np.eye(3)).max() < 1e-14
        assert abs(np.linalg.det(R[i]) - 1) < 1e-14
        qn = q[i] / np.linalg.norm(q[i])
        v = rng.standard_normal(3)
        rv = _hamilton(_hamilton(qn, np.r_[0.0, v]), qn * np.array([1, -1, -1, -1]))[1:]
        assert np.abs(R[i] @ v - rv).max() < 1e-13


def _one(mean, log_scale, quat, logit=0.0, deg=0, rgb_dc=(0.0, 0.0, 0.0)):
    sh = np.zeros((1, (deg + 1) ** 2, 3))
    sh[0, 0] = rgb_dc
    return dict(means=np.array([mean], np.float64), log_scales=np.array([log_scale], np.float64),
                quats=np.array([quat], np.float64), logit_opacity=np.array([logit], np.float64), sh=sh)


def test_projection_isotropic_on_axis_closed_form():
    """Isotropic sigma at (0, 0, z) on the optical axis: Sigma2D = ((f sigma / z)^2 + 0.3) I, mean at the principal point."""
    cams = scenes.identity_camera(64, 48)
    cam = oracle.camera_block(cams, 0)
    f = float(cams.fy[0])
    for z, sig in [(1.0, 0.01), (2.5, 0.03), (7.0, 0.2)]:
        p = oracle.project(_one([0, 0, z], [math.log(sig)] * 3, [0.3, -0.2, 0.5, 0.1]), cam)
        expect = (f * sig / z) ** 2 + 0.3
        a, b, c = p["cov2d"][0]
        assert abs(a - expect) < 1e-10 * expect and abs(c - expect) < 1e-10 * expect and abs(b) < 1e-12
        assert np.allclose(p["xy"][0], [cams.cx[0], cams.cy[0]], atol=1e-12)
        assert p["depth"][0] == pytest.approx(z)
        # both eigenvalues equal: the discriminant is 0, so its floor 0.1 applies
        assert p["radius"][0] == math.ceil(3 * math.sqrt(expect + math.sqrt(0.1)))
        # conic is the inverse
        A, B, C = p["conic"][0]
        assert np.allclose([A, B, C], [1 / expect, 0, 1 / expect], rtol=1e-12, atol=1e-14)


def _numeric_jacobian(cam, t):
    """Central-difference Jacobian of (fx x/z + cx, fy y/z + cy) in camera space."""
    fx, fy, cx, cy = cam[12], cam[13], cam[14], cam[15]
    pi = lambda v: np.array([fx * v[0] / v[2] + cx, fy * v[1] / v[2] + cy])
    J = np.zeros((2, 3))
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (pi(t + e) - pi(t - e)) / (2 * h)
    return J


def test_projection_general_vs_numeric_jacobian():
    """Anisotropic, rotated Gaussians seen by an orbital camera: Sigma2D = J W Sigma W^T J^T + 0.3 I
    with J the numerical Jacobian of the pinhole map, Sigma = R(q) S^2 R(q)^T, conic = inv, radius via eigvalsh."""
    rng = np.random.default_rng(4)
    cams = scenes.front_camera(200, 150, eye=(0.4, -3.0, 1.0))
    cam = oracle.camera_block(cams, 0)
    Rv = cam[:9].reshape(3, 3)
    tv = cam[9:12]
    lim = 1.3 * cam[16]
    checked = 0
    for it in range(200):
        mean = rng.uniform(-0.8, 0.8, 3)
        ls = rng.uniform(-4, -1.5, 3)
        q = rng.standard_normal(4)
        p = oracle.project(_one(mean, ls, q), cam)
        t = Rv @ mean + tv
        if abs(t[0] / t[2]) > lim or abs(t[1] / t[2]) > 1.3 * cam[17]:
            continue
        J = _numeric_jacobian(cam, t)
        Rq = oracle.quat_to_rot(q)[0]
        Sig = Rq @ np.diag(np.exp(2 * ls)) @ Rq.T
        cov = J @ Rv @ Sig @ Rv.T @ J.T + 0.3 * np.eye(2)
        a, b, c = p["cov2d"][0]
        assert np.allclose([a, b, c], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-7, atol=1e-9)
        if p["radius"][0] > 0:
            inv = np.linalg.inv(cov)
            assert np.allclose(p["conic"][0], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-6)
            lam = np.linalg.eigvalsh(cov).max()
            mid = 0.5 * (cov[0, 0] + cov[1, 1])
            if mid * mid - np.linalg.det(cov) > 0.1 + 1e-6:
                assert p["radius"][0] == math.ceil(3 * math.sqrt(lam))
            xy = np.array([cam[12] * t[0] / t[2] + cam[14], cam[13] * t[1] / t[2] + cam[15]])
            assert np.allclose(p["xy"][0], xy, rtol=1e-12)
        checked += 1
    assert checked > 100


def test_projection_monte_carlo_first_order():
    """Sample a tiny 3D Gaussian, project every sample exactly: the sample covariance matches
    J W Sigma W^T J^T (the dilation removed) to first order."""
    rng = np.random.default_rng(5)
    cams = scenes.front_camera(256, 256, eye=(0.3, -2.5, 0.7))
    cam = oracle.camera_block(cams, 0)
    Rv, tv = cam[:9].reshape(3, 3), cam[9:12]
    mean = np.array([0.1, 0.05, -0.1])
    ls = np.log([2e-3, 5e-4, 1e-3])
    q = np.array([0.9, 0.2, -0.3, 0.1])
    p = oracle.project(_one(mean, ls, q), cam)
    Rq = oracle.quat_to_rot(q)[0]
    M = Rq @ np.diag(np.exp(ls))
    X = mean + rng.standard_normal((400000, 3)) @ M.T
    t = X @ Rv.T + tv
    uv = np.stack([cam[12] * t[:, 0] / t[:, 2] + cam[14], cam[13] * t[:, 1] / t[:, 2] + cam[15]], 1)
    S = np.cov(uv.T)
    a, b, c = p["cov2d"][0]
    est = np.array([a - 0.3, b, c - 0.3])
    got = np.array([S[0, 0], S[0, 1], S[1, 1]])
    assert np.abs(est - got).max() < 0.02 * np.abs(est).max()


def test_projection_j_clamp_uses_clamped_ratio():
    """Beyond 1.3 tan(fov/2) the Jacobian is the pinhole Jacobian at the clamped point (x' = 1.3 tan * z)."""
    cams = scenes.identity_camera(64, 64)
    cam = oracle.camera_block(cams, 0)
    lim = 1.3 * cam[16]
    z = 2.0
    x = 1.6 * lim * z
    ls = [math.log(0.05)] * 3
    p = oracle.project(_one([x, 0.0, z], ls, [1, 0, 0, 0]), cam)
    J = _numeric_jacobian(cam, np.array([lim * z, 0.0, z]))
    cov = J @ (np.eye(3) * 0.05 ** 2) @ J.T + 0.3 * np.eye(2)
    assert np.allclose(p["cov2d"][0], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-7)


def test_near_plane_cull():
    cams = scenes.identity_camera(64, 64)
    cam = oracle.camera_block(cams, 0)
    for z, vis in [(0.19, False), (0.2, False), (0.25, True)]:
        p = oracle.project(_one([0, 0, z], [math.log(1e-3)] * 3, [1, 0, 0, 0]), cam)
        assert (p["radius"][0] > 0) == vis


def test_tile_rect_covers_radius_and_clamps():
    """Tiles [x0, x1) contain every pixel centre within r - 1 of the mean in each axis, never leave
    the grid, and tiles = (x1 - x0)(y1 - y0)."""
    rng = np.random.default_rng(6)
    W, H = 100, 70
    TX, TY = 7, 5
    cams = scenes.identity_camera(W, H)
    cam = oracle.camera_block(cams, 0)
    for _ in range(300):
        mean = np.r_[rng.uniform(-1.2, 1.2, 2), rng.uniform(1.0, 3.0)]
        ls = [rng.uniform(-5, -1.5)] * 3
        p = oracle.project(_one(mean, ls, [1, 0, 0, 0]), cam)
        r = p["radius"][0]
        if r == 0:
            continue
        x0, y0, x1, y1 = p["rect"][0]
        assert 0 <= x0 <= x1 <= TX and 0 <= y0 <= y1 <= TY
        assert p["tiles"][0] == (x1 - x0) * (y1 - y0)
        u, v = p["xy"][0]
        for px in range(max(0, math.ceil(u - r + 1)), min(W - 1, math.floor(u + r - 1)) + 1):
            assert x0 <= px // 16 < x1
        for py in range(max(0, math.ceil(v - r + 1)), min(H - 1, math.floor(v + r - 1)) + 1):
            assert y0 <= py // 16 < y1


def test_sh_colour_offset_and_clamp():
    """rgb = Y00 * dc + 0.5, clamped at 0 per channel; the clamp bit records it."""
    cams = scenes.identity_camera(64, 64)
    cam = oracle.camera_block(cams, 0)
    y00 = 0.5 / math.sqrt(math.pi)
    dc = np.array([0.4, -2.0, 0.0]) / y00
    p = oracle.project(_one([0, 0, 2.0], [math.log(0.05)] * 3, [1, 0, 0, 0], rgb_dc=dc), cam)
    assert np.allclose(p["rgb"][0], [0.9, 0.0, 0.5], atol=1e-14)
    assert p["clamp"][0] == 0b010
    assert p["opacity"][0] == pytest.approx(0.5)


def _nearest_f32(q):
    """The float32 nearest to the rational q (ties to the even significand), by exact comparison."""
    from fractions import Fraction
    c = np.float32(float(q))
    cands = [np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))]
    d = [abs(Fraction(float(x)) - q) for x in cands]
    best = min(d)
    ties = [x for x, e in zip(cands, d) if e == best]
    return min(ties, key=lambda x: int(np.float32(x).view(np.uint32)) & 1)


def test_depth_key_is_the_float32_rounding_of_the_exact_depth():
    """The sort key of every Gaussian is the float32 nearest to its exact camera-space z, computed here in
    rational arithmetic from the float32 means and camera."""
    from fractions import Fraction
    rng = np.random.default_rng(11)
    cams = scenes.front_camera(200, 150, eye=(0.4, -3.0, 1.0))
    cam = oracle.camera_block(cams, 0)
    means = rng.uniform(-0.9, 0.9, (400, 3)).astype(np.float32)
    g = dict(means=means.astype(np.float64), log_scales=np.full((400, 3), -3.0), quats=np.tile([1.0, 0, 0, 0], (400, 1)),
             logit_opacity=np.zeros(400), sh=np.zeros((400, 1, 3)))
    p = oracle.project(g, cam)
    R2, t2 = cam[6:9], cam[11]
    for i in range(400):
        z = sum(Fraction(float(R2[j])) * Fraction(float(means[i, j])) for j in range(3)) + Fraction(float(t2))
        assert np.float32(p["depth"][i]) == _nearest_f32(z), i


def test_unstable_flags_rare_on_random_scenes():
    """The float32 near-tie flags mark a small fraction of Gaussians of an ordinary scene."""
    g, cams = scenes.random_scene(3000, 1, 3, 200, 150)
    p = oracle.project({k: np.asarray(v, np.float64) for k, v in g.items()}, oracle.camera_block(cams, 0))
    assert (p["unstable"] != 0).mean() < 2e-3


def test_unstable_flag_radius_at_an_integer():
    """On the axis, 3 sqrt(lambda_max) = k exactly for sigma solving (f sigma / z)^2 + 0.3 + sqrt(0.1) = k^2 / 9:
    the radius decision is flagged; half an integer away it is not."""
    cams = scenes.identity_camera(64, 64)
    cam = oracle.camera_block(cams, 0)
    f, z = float(cams.fy[0]), 2.0
    for k in (4, 7):
        for shift, flag in ((0.0, True), (0.5, False)):
            lam = (k + shift) ** 2 / 9.0
            sig = z / f * math.sqrt(lam - math.sqrt(0.1) - 0.3)
            p = oracle.project(_one([0, 0, z], [math.log(sig)] * 3, [1, 0, 0, 0]), cam)
            assert bool(p["unstable"][0] & 2) == flag, (k, shift)


def test_unstable_flag_rect_at_a_tile_boundary():
    """A splat of radius 16 whose pixel x is an integer u = 32: floor(u - r) / 16 is a tile boundary, so the
    rectangle decision is flagged; at u = 32.3 it is not."""
    cams = scenes.identity_camera(64, 64)
    cam = oracle.camera_block(cams, 0)
    f, cx, z = float(cams.fx[0]), float(cams.cx[0]), 2.0
    sig = z / f * math.sqrt(27.0 - math.sqrt(0.1) - 0.3)  # 3 sqrt(lambda) = 15.59: radius 16
    for u, flag in ((32.0, True), (32.3, False)):
        x = (u - cx) / f * z
        p = oracle.project(_one([x, 0, z], [math.log(sig)] * 3, [1, 0, 0, 0]), cam)
        assert p["radius"][0] == 16
        assert bool(p["unstable"][0] & 4) == flag, u


def test_unstable_flag_near_plane():
    """A mean exactly on the near plane is a flagged cull decision; one well in front of it is not."""
    cams = scenes.identity_camera(64, 64)
    cam = oracle.camera_block(cams, 0)
    for z, flag in ((cam[21], True), (0.25, False)):
        p = oracle.project(_one([0, 0, z], [math.log(1e-3)] * 3, [1, 0, 0, 0]), cam)
        assert bool(p["unstable"][0] & 1) == flag, z
