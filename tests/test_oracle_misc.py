"""Pins of the oracle's optimiser, kNN, ghost filter and learned-init MLP.

* Adam: hand-computed first steps and torch.optim.Adam (float64) over many steps;
* kNN: scipy's cKDTree;
* ghost filter: hand cases of half-open / closed owned boxes;
* bf16 rounding: torch's float64 -> bfloat16 conversion (round to nearest even);
* MLP forward and backward: torch autograd in float64 with the same bf16
  rounding points (rounding applied as a straight-through value change in the
  forward pass, and by gradient hooks on the back-propagated signals).
"""
import math

import numpy as np
import pytest
import torch
from scipy.spatial import cKDTree

import oracle
import synth


def test_adam_first_steps_by_hand():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.1, -3.0, 0.0])
    m = np.zeros(3)
    v = np.zeros(3)
    p1, m1, v1 = oracle.adam(p, g, m, v, 0.01, 0.9, 0.999, 1e-15, 1)
    # t = 1: m_hat = g, v_hat = g^2 -> step = lr * g / (|g| + eps) = lr * sign(g)
    assert np.allclose(p1, [1.0 - 0.01, -2.0 + 0.01, 0.5], atol=1e-12)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)
    g2 = np.array([0.3, 1.0, 0.0])
    p2, m2, v2 = oracle.adam(p1, g2, m1, v1, 0.01, 0.9, 0.999, 1e-15, 2)
    mh = (0.9 * 0.1 * g + 0.1 * g2) / (1 - 0.81)
    vh = (0.999 * 0.001 * g * g + 0.001 * g2 * g2) / (1 - 0.999 ** 2)
    with np.errstate(invalid="ignore", divide="ignore"):
        step = np.where(vh > 0, 0.01 * mh / (np.sqrt(vh) + 1e-15), 0.0)
    assert np.allclose(p2, p1 - step, atol=1e-14)


def test_adam_matches_torch():
    rng = np.random.default_rng(0)
    n = 257
    p = rng.standard_normal(n)
    lr = np.where(np.arange(n) % 3 == 0, 1e-3, 5e-2)
    pt = [torch.tensor(p[lr == a], dtype=torch.float64, requires_grad=True) for a in (1e-3, 5e-2)]
    opt = torch.optim.Adam([{"params": [pt[0]], "lr": 1e-3}, {"params": [pt[1]], "lr": 5e-2}],
                           betas=(0.9, 0.999), eps=1e-15)
    m = np.zeros(n)
    v = np.zeros(n)
    for t in range(1, 31):
        g = rng.standard_normal(n)
        p, m, v = oracle.adam(p, g, m, v, lr, 0.9, 0.999, 1e-15, t)
        opt.zero_grad()
        pt[0].grad = torch.tensor(g[lr == 1e-3])
        pt[1].grad = torch.tensor(g[lr == 5e-2])
        opt.step()
    assert np.allclose(p[lr == 1e-3], pt[0].detach().numpy(), rtol=1e-12, atol=1e-14)
    assert np.allclose(p[lr == 5e-2], pt[1].detach().numpy(), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("k", [3, 16])
def test_knn_matches_kdtree(k):
    pts, _, _ = synth.interface_points(3000, 8, seed=3)
    idx, dist = oracle.knn(pts, k)
    d_ref, i_ref = cKDTree(pts.astype(np.float64)).query(pts.astype(np.float64), k=k + 1)
    assert np.allclose(dist, d_ref[:, 1:], rtol=1e-12, atol=0)
    # indices agree wherever the distances are not tied
    tie = np.zeros_like(idx, bool)
    tie[:, 1:] |= np.isclose(d_ref[:, 2:], d_ref[:, 1:-1], rtol=1e-12)
    tie[:, :-1] |= tie[:, 1:]
    assert np.array_equal(idx[~tie], i_ref[:, 1:][~tie])


def test_owned_filter_cases():
    means = np.array([[0.0, 0.5, 0.5], [0.25, 0.5, 0.5], [0.2499, 0.1, 0.9], [1.0, 0.0, 0.0],
                      [-0.01, 0.5, 0.5], [0.3, 0.5, 0.5]])
    part_of = np.array([0, 0, 0, 1, 0, 1])
    boxes = np.array([[0.0, 0.0, 0.0, 0.25, 1.0, 1.0], [0.25, 0.0, 0.0, 1.0, 1.0, 1.0]])
    closed = np.array([[0, 1, 1], [1, 1, 1]])
    keep = oracle.owned(means, part_of, boxes, closed)
    assert keep.tolist() == [True, False, True, True, False, True]


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(2000) * 10 ** rng.uniform(-6, 6, 2000),
                        [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0]])
    ours = oracle.bf16_round(x)
    ref = torch.tensor(x, dtype=torch.float64).to(torch.bfloat16).to(torch.float64).numpy()
    # torch rounds float64 -> float32 -> bfloat16; compare where that double rounding is harmless
    f32 = x.astype(np.float32).astype(np.float64)
    ok = f32 == x
    assert np.array_equal(ours[ok], ref[ok])
    assert np.abs(ours - ref).max() <= np.abs(x).max() * 2 ** -8


def _mlp_weights(seed):
    s = synth.streams(seed, ["W1", "W2", "W3", "b"])
    return dict(W1=s["W1"].standard_normal((112, 64)) * (2 / 112) ** 0.5,
                b1=s["b"].standard_normal(64) * 0.1,
                W2=s["W2"].standard_normal((64, 64)) * (2 / 64) ** 0.5,
                b2=s["b"].standard_normal(64) * 0.1,
                W3=s["W3"].standard_normal((64, 8)) * (1 / 64) ** 0.5,
                b3=s["b"].standard_normal(8) * 0.1)


def _bf(t):
    return t.to(torch.bfloat16).to(torch.float64)


class _RoundGrad(torch.autograd.Function):
    """Identity forward; rounds the incoming gradient to bf16."""

    @staticmethod
    def forward(ctx, x):
        return x.view_as(x)

    @staticmethod
    def backward(ctx, g):
        return _bf(g)


def _torch_mlp(X, w, T):
    """The same network in torch float64 autograd.  Operands that the definition rounds to bf16
    are rounded with a straight-through value change; back-propagated signals that become GEMM
    operands are rounded by _RoundGrad placed where the oracle rounds them."""
    st = lambda t: t + (_bf(t) - t).detach()
    Xt = torch.tensor(X)
    W = {k: torch.tensor(v, requires_grad=True) for k, v in w.items()}
    a1 = st(Xt) @ st(W["W1"]) + W["b1"]
    h1 = torch.relu(_RoundGrad.apply(a1))
    a2 = st(h1) @ st(W["W2"]) + W["b2"]
    h2 = torch.relu(_RoundGrad.apply(a2))
    y = st(h2) @ st(W["W3"]) + W["b3"]
    y = _RoundGrad.apply(y)
    L = ((y - torch.tensor(T)) ** 2).sum() / (8 * X.shape[0])
    L.backward()
    return float(L.detach()), y.detach().numpy(), {k: v.grad.numpy() for k, v in W.items()}


def test_mlp_matches_torch_autograd():
    rng = np.random.default_rng(1)
    n = 300
    X = np.zeros((n, 112))
    X[:, :99] = rng.standard_normal((n, 99))
    T = rng.standard_normal((n, 8)) * 0.5
    w = _mlp_weights(2)
    f = oracle.mlp_forward(X, w)
    L, g = oracle.mlp_backward(X, w, T)
    Lt, yt, gt = _torch_mlp(X, w, T)
    assert np.allclose(f["Y"], yt, rtol=1e-12, atol=1e-12)
    assert L == pytest.approx(Lt, rel=1e-12)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        # the torch graph rounds d(loss)/dy to bf16 before the W3/b3 gradient, as the oracle does;
        # the ReLU gradient passes where the pre-activation is > 0 in both
        assert np.allclose(g[k], gt[k], rtol=1e-9, atol=1e-12), k


def test_mlp_features_layout():
    pts, nrm, _ = synth.interface_points(500, 4, seed=4)
    idx, dist = oracle.knn(pts, 16)
    X = oracle.mlp_features(pts, nrm, idx, dist)
    i = 17
    dbar = dist[i].mean()
    assert np.allclose(X[i, :48].reshape(16, 3), (pts[idx[i]] - pts[i]) / dbar, rtol=1e-6)
    assert np.allclose(X[i, 48:96].reshape(16, 3), nrm[idx[i]])
    assert np.allclose(X[i, 96:99], nrm[i]) and np.all(X[:, 99:] == 0)
    # offsets have unit mean length by construction
    assert np.linalg.norm(X[:, :48].reshape(-1, 16, 3), axis=2).mean(axis=1) == pytest.approx(1.0, rel=1e-6)


def test_init_gaussians_plain_against_kdtree():
    """Plain initialiser: isotropic log-scale = log of the mean of the 3 nearest-neighbour distances (by
    scipy's cKDTree, self excluded), floored at 1e-7; identity rotation; the default logit opacity."""
    pts, _, _ = synth.interface_points(2000, 8, seed=5)
    pts = pts.astype(np.float64)
    pts[7] = pts[8]  # a duplicate pair ...
    pts[9] = pts[8]  # ... and triple: mean 3-NN distance of point 8's group can be tiny
    d_ref, _ = cKDTree(pts).query(pts, k=4)
    d3 = d_ref[:, 1:].mean(axis=1)
    ls, q, lo = oracle.init_gaussians(d_ref[:, 1:])
    expect = np.log(np.maximum(d3, 1e-7))
    assert np.allclose(ls, np.repeat(expect[:, None], 3, 1), rtol=0, atol=1e-12)
    assert np.array_equal(q, np.tile([1.0, 0, 0, 0], (2000, 1)))
    assert np.allclose(lo, math.log(0.1 / 0.9), rtol=0, atol=1e-15)
    # an all-zero neighbourhood takes the floor
    ls0, _, _ = oracle.init_gaussians(np.zeros((1, 3)))
    assert ls0[0, 0] == pytest.approx(math.log(1e-7), abs=1e-12)


def test_init_gaussians_learned_and_fallback_by_hand():
    """Learned initialiser: log-scale = plain log-scale + outputs 0..2, rotation = outputs 3..6, logit =
    output 7; a Gaussian whose outputs are not all finite, or whose rotation has norm <= 1e-6, keeps the
    plain values."""
    dist = np.array([[0.1, 0.2, 0.3], [0.5, 0.5, 0.5], [1.0, 2.0, 3.0], [0.2, 0.2, 0.2]])
    Y = np.array([[0.1, -0.2, 0.3, 0.5, 0.5, -0.5, 0.5, 1.5],
                  [0.0, 0.0, 0.0, np.nan, 1.0, 0.0, 0.0, 0.0],      # non-finite -> plain
                  [1.0, 1.0, 1.0, 0.0, 0.0, 0.0, 5e-7, -1.0],      # rotation norm 5e-7 -> plain
                  [0.0, 0.0, 0.0, 0.0, 0.0, 2.0, 0.0, np.inf]])     # infinite logit -> plain
    ls, q, lo = oracle.init_gaussians(dist, Y, logit_default=-2.0)
    plain = np.log(dist.mean(axis=1))
    assert np.allclose(ls[0], plain[0] + np.array([0.1, -0.2, 0.3]), atol=1e-14)
    assert np.allclose(q[0], [0.5, 0.5, -0.5, 0.5]) and lo[0] == 1.5
    for i in (1, 2, 3):
        assert np.allclose(ls[i], plain[i], atol=1e-14) and np.array_equal(q[i], [1.0, 0, 0, 0]) and lo[i] == -2.0


def test_mlp_features_hand_configuration_and_invariances():
    """Features of a hand-built neighbourhood (16 neighbours at known offsets), and their behaviour under
    rigid motions and scaling of the whole cloud: offsets and normals rotate with it, translation and
    uniform scaling leave them unchanged."""
    rng = np.random.default_rng(9)
    offs = rng.standard_normal((16, 3))
    offs *= (np.arange(1, 17) / np.linalg.norm(offs, axis=1))[:, None]  # distances 1 .. 16, all distinct
    pts = np.vstack([np.zeros(3), offs])
    nrm = rng.standard_normal((17, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    idx, dist = oracle.knn(pts, 16)
    X = oracle.mlp_features(pts, nrm, idx, dist)
    dbar = np.arange(1, 17).mean()
    assert np.array_equal(idx[0], np.arange(1, 17))
    assert np.allclose(X[0, :48].reshape(16, 3), offs / dbar, atol=1e-14)
    assert np.allclose(X[0, 48:96].reshape(16, 3), nrm[1:], atol=0)
    assert np.allclose(X[0, 96:99], nrm[0], atol=0) and np.all(X[:, 99:] == 0)
    # a rotation, a translation and a scaling of the cloud
    from scipy.spatial.transform import Rotation
    R = Rotation.random(random_state=3).as_matrix()
    p2 = 2.5 * pts @ R.T + np.array([0.3, -1.0, 4.0])
    n2 = nrm @ R.T
    idx2, dist2 = oracle.knn(p2, 16)
    X2 = oracle.mlp_features(p2, n2, idx2, dist2)
    assert np.array_equal(idx2, idx)
    for a, b in ((slice(0, 48), slice(0, 48)), (slice(48, 96), slice(48, 96)), (slice(96, 99), slice(96, 99))):
        rot = X[:, a].reshape(17, -1, 3) @ R.T
        assert np.allclose(X2[:, b].reshape(17, -1, 3), rot, atol=1e-12)
