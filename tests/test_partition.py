"""Host logic of the partitioning (Sec. II, "Data Partitioning"): slabs, ghost layers, owned filter."""
import numpy as np

import oracle
import synth
from paper_2509_12138_gb300.partition import owned_mask, slab_partition


def test_slabs_ghosts_and_ownership():
    pts, _, _ = synth.interface_points(20000, 8, seed=1)
    part = slab_partition(pts, 8, 0.05)
    x = pts[:, 0].astype(np.float64)
    order = part.order
    assert part.offsets[-1] == len(order)
    w = 1.0 / 8
    owner = np.minimum((x / w).astype(int), 7)
    # every point appears in its own slab's partition
    for i in np.random.default_rng(0).choice(len(pts), 500, replace=False):
        k = owner[i]
        assert i in set(part.members[k].tolist())
    # members lie in the slab widened by the ghost layer on interior sides only
    for k in range(8):
        xm = x[part.members[k]]
        lo = part.edges[k] - (0.05 * w if k > 0 else 0)
        hi = part.edges[k + 1] + (0.05 * w if k < 7 else 0)
        assert xm.min() >= lo - 1e-12 and xm.max() <= hi + 1e-12
    # ghost copies: points within 0.05 w of an interior cut appear twice
    dist = np.min(np.abs(x[:, None] - part.edges[None, 1:8]), axis=1)
    near, far = dist < 0.05 * w * 0.999, dist > 0.05 * w * 1.001
    counts = np.bincount(order, minlength=len(pts))
    assert np.all(counts[far] == 1) and np.all(counts[near] == 2)
    # the owned filter keeps exactly one copy of every point (untrained means)
    keep = owned_mask(pts[order], part)
    assert np.array_equal(np.bincount(order[keep], minlength=len(pts)), np.ones(len(pts), int))


def test_owned_filter_matches_oracle():
    pts, _, _ = synth.interface_points(5000, 4, seed=2)
    part = slab_partition(pts, 5, 0.1)
    means = pts[part.order] + np.random.default_rng(1).normal(0, 0.01, (len(part.order), 3)).astype(np.float32)
    part_of = np.repeat(np.arange(part.n), part.sizes())
    ref = oracle.owned(means, part_of, part.boxes, part.closed_hi)
    assert np.array_equal(owned_mask(means, part), ref)


def test_uneven_slab_populations():
    counts = [500, 1500, 2500, 3500, 4000, 4500, 5500, 6000]
    pts, _, _ = synth.slab_density_points(8, counts, seed=3)
    part = slab_partition(pts, 8, 0.0)
    assert np.array_equal(part.sizes(), counts)


def test_spatial_order_is_the_z_order():
    """synth.spatial_order sorts points by their Morton code on a 1024^3 grid over the bounding box
    (checked against a bit-by-bit interleave), stably, and is a permutation."""
    rng = np.random.default_rng(7)
    p = rng.random((3000, 3))
    p[:20] = p[20:40]  # equal points keep their order
    o = synth.spatial_order(p)
    assert np.array_equal(np.sort(o), np.arange(len(p)))
    lo, hi = p.min(0), p.max(0)
    q = np.round((p - lo) / (hi - lo) * 1023).astype(np.int64)
    code = np.zeros(len(p), np.int64)
    for b in range(10):
        for a in range(3):
            code |= ((q[:, a] >> b) & 1) << (3 * b + a)
    assert np.array_equal(o, np.argsort(code, kind="stable"))


def test_device_z_order_bits():
    """The 100M render scene's (x, y) Z-order key: 16-bit quantised coordinates with their bits
    interleaved (x on even, y on odd positions), checked bit by bit."""
    import torch
    from paper_2509_12138_gb300.workload import _spread2
    v = torch.rand(500, generator=torch.Generator().manual_seed(3))
    q = (v.double() * 65535.0).round().long()
    got = _spread2(v)
    for i in range(len(v)):
        want = 0
        for b in range(16):
            want |= ((int(q[i]) >> b) & 1) << (2 * b)
        assert int(got[i]) == want
    key = _spread2(v[:250]) | (_spread2(v[250:]) << 1)
    assert int(key.max()) < 1 << 32
