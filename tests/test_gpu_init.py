"""kNN, the MLP (features, forward, training gradients) and the initialisers vs the oracle (GPU)."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2509_12138_gb300 import init as gi

pytestmark = pytest.mark.gpu


def _surface(n, seed, modes=8):
    pts, nrm, _ = synth.interface_points(n, modes, seed)
    return pts, nrm


@pytest.mark.parametrize("n,k,seed", [(20000, 16, 0), (20000, 3, 1), (3000, 8, 2), (17, 16, 3)])
def test_knn_matches_bruteforce(n, k, seed):
    pts, _ = _surface(n, seed)
    idx, dist = gi.knn(torch.from_numpy(pts).cuda(), k)
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    oi, od = oracle.knn(pts, k)
    finite = np.isfinite(od)
    assert np.array_equal(np.isfinite(dist), finite)
    assert np.allclose(dist[finite], od[finite], rtol=2e-6, atol=1e-7)
    # indices: equal except where FP32 and FP64 distances nearly tie (rank swap)
    near = np.zeros_like(finite)
    rel = np.abs(np.diff(od, axis=1)) <= 1e-6 * np.maximum(od[:, 1:], 1e-30)
    near[:, 1:] |= rel
    near[:, :-1] |= rel
    ok = finite & ~near
    assert np.array_equal(idx[ok], oi[ok])
    assert (near & finite).mean() < 1e-3


def test_mlp_features_match_oracle():
    pts, nrm = _surface(5000, 4)
    P, Nn = torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda()
    idx, dist = gi.knn(P, 16)
    X = gi.mlp_features(P, Nn, idx, dist).cpu().numpy().view(np.uint16)
    Xf = (X.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    ref = oracle.bf16_round(oracle.mlp_features(pts, nrm, idx.cpu().numpy(), dist.cpu().numpy()))
    # bf16 of the same value; FP32 vs FP64 arithmetic may flip a rounding at a bf16 midpoint
    diff = np.abs(Xf - ref)
    ulp = np.abs(ref) * 2 ** -7 + 1e-30
    assert np.all(diff <= ulp)
    assert (diff > 0).mean() < 1e-3


def _weights(seed):
    w = gi.init_weights(seed).cpu().numpy()
    g = np.random.default_rng(seed + 1)
    w[11392:11392 + 512] = g.standard_normal(512) * 0.1  # non-zero last layer
    w[7168:7232] = g.standard_normal(64) * 0.1
    return w


def _split(w):
    return dict(W1=w[0:7168].reshape(112, 64), b1=w[7168:7232], W2=w[7232:11328].reshape(64, 64),
                b2=w[11328:11392], W3=w[11392:11904].reshape(64, 8), b3=w[11904:11912])


def test_mlp_forward_matches_oracle():
    pts, nrm = _surface(6000, 5)
    P, Nn = torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda()
    idx, dist = gi.knn(P, 16)
    w = _weights(3)
    Y = gi.mlp_forward(torch.from_numpy(w).cuda(), P, Nn, idx, dist).cpu().numpy()
    X = oracle.mlp_features(pts, nrm, idx.cpu().numpy(), dist.cpu().numpy())
    ref = oracle.mlp_forward(X, _split(w.astype(np.float64)))["Y"]
    err = np.abs(Y - ref)
    # fp32 accumulation + occasional one-ulp bf16 flips of intermediates
    assert np.median(err) <= 1e-5 * np.abs(ref).max()
    assert err.max() <= 2e-2 * np.abs(ref).max()


def test_mlp_train_step_gradients_match_oracle():
    pts, nrm = _surface(4000, 6)
    P, Nn = torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda()
    idx, dist = gi.knn(P, 16)
    w = _weights(4)
    T = np.random.default_rng(0).standard_normal((4000, 8)).astype(np.float32) * 0.3
    tr = gi.MLPTrainer(torch.from_numpy(w).cuda(), lr=1e-3)
    loss = float(tr.step(P, Nn, idx, dist, torch.from_numpy(T).cuda()).item())
    g = tr.grad.cpu().numpy()
    X = oracle.mlp_features(pts, nrm, idx.cpu().numpy(), dist.cpu().numpy())
    L, gr = oracle.mlp_backward(X, _split(w.astype(np.float64)), T.astype(np.float64))
    assert loss == pytest.approx(L, rel=1e-3)
    flat = np.concatenate([gr[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
    for sl in (slice(0, 7168), slice(7168, 7232), slice(7232, 11328), slice(11328, 11392), slice(11392, 11904),
               slice(11904, 11912)):
        sc = np.abs(flat[sl]).max()
        assert np.abs(g[sl] - flat[sl]).max() <= 2e-2 * sc
    # Adam applied: first step moves each weight with a non-zero gradient by lr
    w1 = tr.w.cpu().numpy()
    moved = np.abs(w1 - w)
    nz = np.abs(g) > 1e-5
    assert np.allclose(moved[nz], 1e-3, rtol=1e-2)


def test_mlp_training_reduces_loss():
    pts, nrm = _surface(20000, 7)
    P, Nn = torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda()
    idx, dist = gi.knn(P, 16)
    # a learnable target: the normal's rotation and a scale offset from the normal's tilt
    q = torch.from_numpy(synth.surfel_quats(nrm)).cuda()
    T = torch.cat([-0.5 * Nn[:, 2:3].repeat(1, 3), q, torch.full((20000, 1), 0.3, device="cuda")], dim=1).contiguous()
    tr = gi.MLPTrainer(gi.init_weights(0), lr=3e-3)
    first = float(tr.step(P, Nn, idx, dist, T).item())
    for _ in range(300):
        last = tr.step(P, Nn, idx, dist, T)
    assert float(last.item()) < 0.2 * first


def test_plain_and_learned_init_match_oracle():
    pts, nrm = _surface(8000, 8)
    P, Nn = torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda()
    n = len(pts)
    params = torch.zeros((4, n, 4), device="cuda")
    gi.init_gaussians(params, P)
    idx3, d3 = gi.knn(P, 3)
    ls, q, lo = oracle.init_gaussians(d3.cpu().numpy())
    a = params.cpu().numpy()
    assert np.allclose(a[0, :, :3], pts) and np.allclose(a[1, :, :3], ls, atol=1e-5)
    assert np.allclose(a[2], q) and np.allclose(a[1, :, 3], lo)
    # learned form
    w = _weights(9)
    idx, dist = gi.knn(P, 16)
    params2 = torch.zeros((4, n, 4), device="cuda")
    gi.init_gaussians(params2, P, Nn, torch.from_numpy(w).cuda(), idx, dist)
    Y = gi.mlp_forward(torch.from_numpy(w).cuda(), P, Nn, idx, dist).cpu().numpy()
    ls2, q2, lo2 = oracle.init_gaussians(dist.cpu().numpy(), Y)
    b = params2.cpu().numpy()
    assert np.allclose(b[1, :, :3], ls2, atol=1e-5) and np.allclose(b[2], q2, atol=1e-6)
    assert np.allclose(b[1, :, 3], lo2, atol=1e-6)
    # fallback: NaN weights give the plain values
    wn = w.copy()
    wn[11904:] = np.nan
    params3 = torch.zeros((4, n, 4), device="cuda")
    gi.init_gaussians(params3, P, Nn, torch.from_numpy(wn).cuda(), idx, dist)
    c = params3.cpu().numpy()
    ls3, q3, lo3 = oracle.init_gaussians(dist.cpu().numpy())
    assert np.allclose(c[1, :, :3], ls3, atol=1e-5) and np.allclose(c[2], q3)
