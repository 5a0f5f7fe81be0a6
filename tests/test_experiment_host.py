"""Host logic of the experiments (CPU): the MLP fit's random-subset reordering."""
import torch

from paper_2509_12138_gb300 import experiment as X


def test_subset_first_keeps_each_point_and_its_neighbours():
    g = torch.Generator().manual_seed(0)
    n, k = 500, 16
    P = torch.rand((n, 3), generator=g)
    Nn = torch.rand((n, 3), generator=g)
    idx = torch.randint(0, n, (n, k), generator=g, dtype=torch.int32)
    dist = torch.rand((n, k), generator=g)
    tg = torch.rand((n, 8), generator=g)
    P2, N2, i2, d2, t2 = X.subset_first(P, Nn, idx, dist, tg, seed=3)
    assert i2.dtype == idx.dtype and i2.shape == idx.shape
    # the rows are a permutation of the points, each with its own normal, distances and targets
    order = torch.stack([torch.nonzero((P == p).all(1))[0, 0] for p in P2])
    assert sorted(order.tolist()) == list(range(n))
    assert torch.equal(N2, Nn[order]) and torch.equal(d2, dist[order]) and torch.equal(t2, tg[order])
    # row r's neighbour j is, in the new numbering, the same point as before
    assert torch.equal(P2[i2.long()], P[idx[order].long()])
    # seeded: the same order every time
    assert torch.equal(X.subset_first(P, Nn, idx, dist, tg, seed=3)[0], P2)
