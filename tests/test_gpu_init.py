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


U32 = 2.0 ** -24  # unit roundoff of float32


def _oracle_knn(pts, k):
    """The oracle's exact neighbours and their float32 distances (fed to both sides)."""
    oi, od = oracle.knn(pts, k)
    return oi, od.astype(np.float32)


def _dev(pts, nrm, oi, od):
    return (torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda(),
            torch.from_numpy(oi.astype(np.int32)).cuda(), torch.from_numpy(od).cuda())


def _flip(v, err):
    """True where a value within err of v may round to another bfloat16 than v itself does."""
    return oracle.bf16_round(v - err) != oracle.bf16_round(v + err)


def test_mlp_features_match_oracle():
    """The kernels' bf16 features equal the bf16 rounding of the oracle's, except offsets whose value lies
    within the float32 error of the kernel's arithmetic (difference and division of float32 values, mean of
    16 float32 distances: 32 ulp) of a bf16 rounding boundary; those are counted."""
    pts, nrm = _surface(5000, 4)
    oi, od = _oracle_knn(pts, 16)
    P, Nn, idx, dist = _dev(pts, nrm, oi, od)
    X = gi.mlp_features(P, Nn, idx, dist).cpu().numpy().view(np.uint16)
    Xf = (X.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    Xo = oracle.mlp_features(pts, nrm, oi, od.astype(np.float64))
    ref = oracle.bf16_round(Xo)
    risky = np.zeros_like(Xo, bool)
    risky[:, :48] = _flip(Xo[:, :48], 32 * U32 * np.abs(Xo[:, :48]))
    assert np.array_equal(Xf[~risky], ref[~risky])
    assert risky.mean() < 1e-3
    print(f"features: {int(risky.sum())} of {risky.size} values near a bf16 rounding boundary")


def _weights(seed):
    w = gi.init_weights(seed).cpu().numpy()
    g = np.random.default_rng(seed + 1)
    w[11392:11392 + 512] = g.standard_normal(512) * 0.1  # non-zero last layer
    w[7168:7232] = g.standard_normal(64) * 0.1
    return w


def _split(w):
    return dict(W1=w[0:7168].reshape(112, 64), b1=w[7168:7232], W2=w[7232:11328].reshape(64, 64),
                b2=w[11328:11392], W3=w[11392:11904].reshape(64, 8), b3=w[11904:11912])


def _rdiff(x, dx, relu=False):
    """Largest |bf16(g(x')) - bf16(g(x))| over |x' - x| <= dx, g the identity or the ReLU (both monotone):
    0 unless a rounding boundary lies within dx of x."""
    g = (lambda t: np.maximum(t, 0.0)) if relu else (lambda t: t)
    mid = oracle.bf16_round(g(x))
    return np.maximum(oracle.bf16_round(g(x + dx)) - mid, mid - oracle.bf16_round(g(x - dx)))


def _acc(K, *terms):
    """Bound of the kernels' float32 accumulation of a K-term product sum (products exact in float32):
    4 (K + 1) 2^-24 sum |a b| (the factor 4 leaves room for the tensor cores' accumulation order)."""
    return 4 * (K + 1) * U32 * sum(terms)


def _forward_bounds(Xo, Wd):
    """The oracle's forward and a bound on the kernels' deviation from it, propagated layer by layer: the
    offset features may differ by 32 float32 ulp before their bf16 rounding; each layer adds its float32
    accumulation error to the deviation its inputs carry, and each bf16 rounding of a (ReLU-ed) activation
    turns the deviation into the largest change of the rounded value (_rdiff), which is 0 unless a rounding
    boundary lies within reach.  Returns the forward, the output bound dY [n, 8], the per-unit bounds and
    a flag per point: some rounding of its chain may go the other way."""
    f = oracle.mlp_forward(Xo, Wd)
    Wb = {k: oracle.bf16_round(Wd[k]) for k in ("W1", "W2", "W3")}
    aW1, aW2, aW3 = np.abs(Wb["W1"]), np.abs(Wb["W2"]), np.abs(Wb["W3"])
    Xb, H1b, H2b = oracle.bf16_round(Xo), oracle.bf16_round(f["H1"]), oracle.bf16_round(f["H2"])
    dXb = np.zeros_like(Xo)
    dXb[:, :48] = _rdiff(Xo[:, :48], 32 * U32 * np.abs(Xo[:, :48]))
    dA1 = dXb @ aW1 + _acc(112, (np.abs(Xb) + dXb) @ aW1, np.abs(Wd["b1"]))
    dH1 = _rdiff(f["A1"], dA1, relu=True)
    dA2 = dH1 @ aW2 + _acc(64, (np.abs(H1b) + dH1) @ aW2, np.abs(Wd["b2"]))
    dH2 = _rdiff(f["A2"], dA2, relu=True)
    dY = dH2 @ aW3 + _acc(64, (np.abs(H2b) + dH2) @ aW3, np.abs(Wd["b3"]))
    flag = (dXb > 0).any(axis=1) | (dH1 > 0).any(axis=1) | (dH2 > 0).any(axis=1)
    return f, dY, flag, dict(Xb=Xb, H1b=H1b, H2b=H2b, Wb=Wb, dXb=dXb, dA1=dA1, dH1=dH1, dA2=dA2, dH2=dH2)


def test_mlp_forward_matches_oracle():
    """Every output within the propagated bound of the kernels' float32 accumulation and of the bf16
    roundings that may go the other way; the points where one may are counted."""
    pts, nrm = _surface(6000, 5)
    oi, od = _oracle_knn(pts, 16)
    P, Nn, idx, dist = _dev(pts, nrm, oi, od)
    w = _weights(3)
    Y = gi.mlp_forward(torch.from_numpy(w).cuda(), P, Nn, idx, dist).cpu().numpy()
    Xo = oracle.mlp_features(pts, nrm, oi, od.astype(np.float64))
    f, dY, flag, _ = _forward_bounds(Xo, _split(w.astype(np.float64)))
    err = np.abs(Y - f["Y"])
    print(f"forward: {int(flag.sum())} of {len(flag)} points where a bf16 rounding may go the other way; "
          f"largest error / bound {(err / dY).max():.3f}; median error {np.median(err):.2e}")
    assert np.all(err <= dY)


def test_mlp_train_step_gradients_match_oracle():
    """One training step: the loss and every weight gradient within the bound propagated through the
    backward pass (the output signal's and the back-propagated signals' bf16 roundings, the ReLU masks of
    units whose pre-activation lies within its bound of 0, and the float32 accumulation over the points,
    4 (n + 64) 2^-24 sum_i |a_i| |b_i|)."""
    pts, nrm = _surface(4000, 6)
    n = len(pts)
    oi, od = _oracle_knn(pts, 16)
    P, Nn, idx, dist = _dev(pts, nrm, oi, od)
    w = _weights(4)
    Wd = _split(w.astype(np.float64))
    T = np.random.default_rng(0).standard_normal((n, 8)).astype(np.float32) * 0.3
    tr = gi.MLPTrainer(torch.from_numpy(w).cuda(), lr=1e-3)
    loss = float(tr.step(P, Nn, idx, dist, torch.from_numpy(T).cuda()).item())
    g = tr.grad.cpu().numpy()
    Xo = oracle.mlp_features(pts, nrm, oi, od.astype(np.float64))
    L, gr = oracle.mlp_backward(Xo, Wd, T.astype(np.float64))
    f, dY, flag, b = _forward_bounds(Xo, Wd)
    aW2, aW3 = np.abs(b["Wb"]["W2"]), np.abs(b["Wb"]["W3"])
    scale = 1.0 / (8.0 * n)
    e = f["Y"] - T
    # loss: outputs within dY, float32 accumulation of n * 8 squares
    assert abs(loss - L) <= 4 * (n + 64) * U32 * L + ((2 * np.abs(e) * dY + dY * dY).sum()) * scale
    # output signal 2 (Y - T) / (8 n) and its bf16 rounding
    v = 2.0 * e * scale
    dyb = oracle.bf16_round(v)
    ddy = _rdiff(v, 2.0 * scale * dY + 4 * U32 * np.abs(v))
    # dH2 = bf16(mask(A2 > 0) (dY W3^T)): a mask that may flip lets the value change by all of it
    a2 = dyb @ b["Wb"]["W3"].T
    da2 = ddy @ aW3.T + _acc(8, (np.abs(dyb) + ddy) @ aW3.T)
    flip2 = np.abs(f["A2"]) <= b["dA2"]
    d2v = np.where(f["A2"] > 0, a2, 0.0)
    dh2b = oracle.bf16_round(d2v)
    ddh2 = np.where(flip2, np.abs(dh2b) + _rdiff(d2v, da2) + da2 + np.abs(a2), _rdiff(d2v, np.where(f["A2"] > 0, da2, 0.0)))
    a1 = dh2b @ b["Wb"]["W2"].T
    da1 = ddh2 @ aW2.T + _acc(64, (np.abs(dh2b) + ddh2) @ aW2.T)
    flip1 = np.abs(f["A1"]) <= b["dA1"]
    d1v = np.where(f["A1"] > 0, a1, 0.0)
    dh1b = oracle.bf16_round(d1v)
    ddh1 = np.where(flip1, np.abs(dh1b) + _rdiff(d1v, da1) + da1 + np.abs(a1), _rdiff(d1v, np.where(f["A1"] > 0, da1, 0.0)))
    # weight gradients: sums over points of (activation) x (signal); each factor within its bound
    gam = 4 * (n + 64) * U32

    def wb(act, dact, sig, dsig):
        return (dact.T @ np.abs(sig) + np.abs(act).T @ dsig + dact.T @ dsig
                + gam * (np.abs(act) + dact).T @ (np.abs(sig) + dsig))

    bound = np.concatenate([wb(b["Xb"], b["dXb"], dh1b, ddh1).reshape(-1),
                            (ddh1 + gam * (np.abs(dh1b) + ddh1)).sum(0),
                            wb(b["H1b"], b["dH1"], dh2b, ddh2).reshape(-1),
                            (ddh2 + gam * (np.abs(dh2b) + ddh2)).sum(0),
                            wb(b["H2b"], b["dH2"], dyb, ddy).reshape(-1),
                            (ddy + gam * (np.abs(dyb) + ddy)).sum(0)])
    flat = np.concatenate([gr[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
    err = np.abs(g - flat)
    flagged = flag | (ddy > 0).any(axis=1) | (ddh2 > 0).any(axis=1) | (ddh1 > 0).any(axis=1)
    print(f"train step: {int(flagged.sum())} of {n} points where a bf16 rounding may go the other way; "
          f"largest gradient error / bound {(err / np.maximum(bound, 1e-300)).max():.3f}")
    assert np.all(err <= bound)
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
    gi.init_gaussians(params, P)  # the kernels' own 3-NN
    _, d3 = oracle.knn(pts, 3)
    ls, q, lo = oracle.init_gaussians(d3)
    a = params.cpu().numpy()
    # float32 distances of the same neighbours (a near-tie swap leaves the mean distance unchanged)
    assert np.allclose(a[0, :, :3], pts) and np.allclose(a[1, :, :3], ls, atol=1e-5)
    assert np.allclose(a[2], q) and np.allclose(a[1, :, 3], lo)
    # learned form: the oracle's neighbours on both sides, the oracle's network outputs on its side
    w = _weights(9)
    oi, od = _oracle_knn(pts, 16)
    _, _, idx, dist = _dev(pts, nrm, oi, od)
    params2 = torch.zeros((4, n, 4), device="cuda")
    gi.init_gaussians(params2, P, Nn, torch.from_numpy(w).cuda(), idx, dist)
    fo, dY, _, _ = _forward_bounds(oracle.mlp_features(pts, nrm, oi, od.astype(np.float64)),
                                   _split(w.astype(np.float64)))
    ls2, q2, lo2 = oracle.init_gaussians(od.astype(np.float64), fo["Y"])
    b = params2.cpu().numpy()
    # log-scale: log d3 (float32) + output; rotation, logit: the outputs, within the output bound (rotation
    # and logit are stored as computed; the fallback applies to no point here)
    assert np.all(np.abs(b[1, :, :3] - ls2) <= dY[:, :3] + 1e-5)
    assert np.all(np.abs(b[2] - q2) <= dY[:, 3:7] + 1e-7)
    assert np.all(np.abs(b[1, :, 3] - lo2) <= dY[:, 7] + 1e-7)
    # fallback: NaN weights give the plain values
    wn = w.copy()
    wn[11904:] = np.nan
    params3 = torch.zeros((4, n, 4), device="cuda")
    gi.init_gaussians(params3, P, Nn, torch.from_numpy(wn).cuda(), idx, dist)
    c = params3.cpu().numpy()
    ls3, q3, lo3 = oracle.init_gaussians(od.astype(np.float64))
    assert np.allclose(c[1, :, :3], ls3, atol=1e-5) and np.allclose(c[2], q3)
