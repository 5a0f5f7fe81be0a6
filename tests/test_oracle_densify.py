"""Pins of the density-control oracle (oracle/densify.py) against closed forms, scipy and hand-built cases."""
import math

import numpy as np
import pytest

from oracle import densify as D


def test_rotation_matches_scipy():
    R_ = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(0)
    for _ in range(20):
        q = rng.normal(size=4)  # (w, x, y, z), not normalised
        ref = R_.from_quat(np.r_[q[1:], q[0]] / np.linalg.norm(q)).as_matrix()  # scipy: scalar last
        np.testing.assert_allclose(D.quat_rot(q), ref, atol=1e-12)


def test_stats_closed_form():
    ga, dn, mr = D.stats(np.zeros(3), np.zeros(3), np.zeros(3), [(1e-4, 2e-4), (5e-5, 0.0), (1.0, 1.0)],
                         [3, 7, 0], 200, 100)
    assert ga[0] == pytest.approx(math.hypot(1e-4 * 100, 2e-4 * 50))
    assert ga[1] == pytest.approx(5e-5 * 100)
    assert ga[2] == 0.0 and dn.tolist() == [1.0, 1.0, 0.0] and mr.tolist() == [3.0, 7.0, 0.0]


def _case():
    logit = lambda o: math.log(o / (1 - o))
    g = {"means": np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [3, 0, 0], [4, 0, 0], [5, 0, 0]], float),
         "log_scales": np.log(np.array([[0.001] * 3, [0.001] * 3, [0.002, 0.001, 0.001], [0.05, 0.02, 0.01],
                                        [0.001] * 3, [0.001] * 3])),
         "quats": np.array([[1, 0, 0, 0], [1, 0, 0, 0], [1, 0, 0, 0], [0.9, 0.1, -0.3, 0.2], [1, 0, 0, 0],
                            [1, 0, 0, 0]], float),
         "logit_opacity": np.array([logit(0.0025), logit(0.5), logit(0.5), logit(0.7), logit(0.5), logit(0.5)]),
         "sh": np.arange(6 * 4 * 3, dtype=float).reshape(6, 4, 3)}
    # g0 low opacity, g1 small gradient, g2 clone, g3 split, g4 too large on screen, g5 never seen
    grad = np.array([1.0, 1e-5, 1.0, 1.0, 1.0, 0.0])
    denom = np.array([1.0, 1.0, 2.0, 1.0, 1.0, 0.0])
    maxr = np.array([2.0, 2.0, 2.0, 2.0, 25.0, 0.0])
    return g, grad, denom, maxr


def test_plan_hand_case():
    g, grad, denom, maxr = _case()
    act = D.plan(g, grad, denom, maxr, step=3500, extent=1.0)
    assert act.tolist() == [0, 1, 2, 3, 0, 1]
    # before the first opacity reset, the screen-size rule is off: g4 is cloned instead
    assert D.plan(g, grad, denom, maxr, step=1000, extent=1.0).tolist() == [0, 1, 2, 3, 2, 1]
    # the clone / split boundary is percent_dense x extent on the largest scale
    assert D.plan(g, grad, denom, maxr, step=1000, extent=0.1)[2] == 3


def test_apply_hand_case():
    g, grad, denom, maxr = _case()
    act = np.array([0, 1, 2, 3, 0, 1])
    m = {k: np.asarray(a, float) + 1.0 for k, a in g.items()}
    v = {k: np.asarray(a, float) + 2.0 for k, a in g.items()}
    z = np.random.default_rng(1).normal(size=(6, 2, 3))
    out, om, ov = D.apply(g, m, v, act, z)
    # order: survivors g1, g2, g5; the copy of g2; the two children of g3
    assert out["means"][:, 0].tolist()[:4] == [1.0, 2.0, 5.0, 2.0] and len(out["means"]) == 6
    for k in g:
        np.testing.assert_array_equal(out[k][3], g[k][2])          # copy is exact
        np.testing.assert_array_equal(om[k][1], m[k][2])           # survivors keep their moments
        assert not np.any(om[k][3:]) and not np.any(ov[k][3:])      # new Gaussians start from zero moments
    s = np.exp(g["log_scales"][3])
    R = pytest.importorskip("scipy.spatial.transform").Rotation.from_quat(
        np.r_[g["quats"][3][1:], g["quats"][3][0]] / np.linalg.norm(g["quats"][3])).as_matrix()
    for k in range(2):
        np.testing.assert_allclose(out["means"][4 + k], g["means"][3] + R @ (s * z[3, k]), atol=1e-12)
        np.testing.assert_allclose(np.exp(out["log_scales"][4 + k]), s / 1.6, rtol=1e-12)
        np.testing.assert_array_equal(out["sh"][4 + k], g["sh"][3])
        assert out["logit_opacity"][4 + k] == g["logit_opacity"][3]


def test_split_children_sample_the_gaussian():
    """Children are draws from the source Gaussian itself: their mean offsets have covariance R S^2 R^T."""
    n = 60000
    q = np.array([0.8, 0.3, -0.4, 0.2])
    s = np.array([0.3, 0.1, 0.05])
    g = {"means": np.zeros((n, 3)), "log_scales": np.tile(np.log(s), (n, 1)), "quats": np.tile(q, (n, 1)),
         "logit_opacity": np.zeros(n), "sh": np.zeros((n, 1, 3))}
    z = np.random.default_rng(2).normal(size=(n, 2, 3))
    out, _, _ = D.apply(g, g, g, np.full(n, 3), z)
    cov = np.cov(out["means"].T)
    R = D.quat_rot(q)
    np.testing.assert_allclose(cov, R @ np.diag(s * s) @ R.T, atol=0.02 * s.max() ** 2)


def test_opacity_reset():
    g = {"logit_opacity": np.array([-6.0, 0.0, 3.0]), "means": np.zeros((3, 3))}
    m = {"logit_opacity": np.ones(3), "means": np.ones((3, 3))}
    g2, m2, v2 = D.opacity_reset(g, m, m)
    lim = math.log(0.01 / 0.99)
    assert g2["logit_opacity"].tolist() == [-6.0, lim, lim]
    assert not np.any(m2["logit_opacity"]) and not np.any(v2["logit_opacity"]) and np.all(m2["means"] == 1)
