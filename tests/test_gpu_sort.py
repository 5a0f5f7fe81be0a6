"""The three sort designs give the same lists (needs a GPU).

gs_bin_sort sorts the visible records by depth (stable radix passes over 32-bit depth keys), emits their tile
instances in that order and bins them with a stable sort on (unit | tile); gs_bin_sort_global sorts all
(unit | tile | depth) instance keys with one global stable radix sort; gs_bin_sort_bucketed gathers the tile
instances per (unit, tile) list with atomics and sorts each list on its own (one CTA in shared memory for
lists of up to 4096 instances, 4096-key jobs of multi-CTA radix passes for longer ones; runs of equal depth
ordered by record index).  All must give bit-identical sorted record ids, tile ranges, instance counts and
block masks, and (through the parity tests) the oracle's lists."""
import numpy as np
import pytest
import torch

import paper_2509_12138_gb300 as gs
import synth
from tests import scenes

pytestmark = pytest.mark.gpu

DESIGNS = ("bucketed", "global", "depth_first")


def _all(g, cams, deg, units=None, chunk=1024, cap=None, masks=True):
    n = g["means"].shape[0]
    units = units or gs.Units.single(n, len(cams))
    fr = gs.Frame(n, units, cams.width, cams.height, deg, with_backward=False, with_loss=False, chunk=chunk,
                  max_instances=cap)
    fr.use_masks = masks  # False: no schedule, so no block masks
    params = gs.pack_params(g, deg)
    camd = gs.pack_cameras(cams)
    if cap is None:
        fr.fit_capacity(params, camd)
    out = []
    for design in DESIGNS:
        fr.preprocess(params, camd)
        fr.sort(design)
        torch.cuda.synchronize()
        st = fr.read_status()
        I = fr.instances()
        out.append(dict(status=st, I=I, vals=fr.sorted_vals[:I].cpu().numpy().copy(),
                        ranges=fr.ranges.cpu().numpy().copy(), masks=fr.block_masks[:I].cpu().numpy().copy()))
    return out


def _same(*outs, masks=True):
    a = outs[0]
    for b in outs[1:]:
        assert a["status"] == b["status"] == 0
        assert a["I"] == b["I"] > 0
        assert np.array_equal(a["ranges"], b["ranges"])
        assert np.array_equal(a["vals"], b["vals"])
        if masks:
            assert np.array_equal(a["masks"], b["masks"])


@pytest.mark.parametrize("n,deg,W,H,seed", [(3000, 3, 200, 150, 0), (20000, 0, 333, 97, 1), (1, 0, 64, 64, 2)])
def test_bucketed_sort_equals_global_sort(n, deg, W, H, seed):
    g, cams = scenes.random_scene(n, deg, seed, W, H)
    a, b, c = _all(g, cams, deg)
    _same(a, b, c)


def test_bucketed_sort_multi_unit():
    g = synth.random_gaussians(4000, 1, 7, extent=0.7, log_scale_range=(-3.2, -2.0))
    cams = synth.orbital_cameras(3, 3.0, width=150, height=110)
    a, b, c = _all(g, cams, 1)
    _same(a, b, c)


def test_bucketed_sort_long_lists():
    """Lists of ~8,400 entries (more than a CTA sorts in shared memory: multi-CTA passes)."""
    g, cams = scenes.deep_stop_scene(3, W=32, H=32, n_faint=2100, fillers_per_tile=6300, deg=0)
    a, b, c = _all(g, cams, 0)
    _same(a, b, c)
    lens = a["ranges"][:, 1] - a["ranges"][:, 0]
    assert lens.max() > 4096


def _level_scene(per_tile, levels, seed):
    """16 * per_tile Gaussians of 1.5 px over a 64x64 identity view, their depths drawn from `levels` values
    (levels = 1: one depth), so every list is made of runs of equal depth."""
    rng = np.random.default_rng(seed)
    cams = scenes.identity_camera(64, 64)
    f, cx = float(cams.fx[0]), float(cams.cx[0])
    n = 16 * per_tile
    z = rng.choice(np.linspace(2.0, 3.0, levels), n) if levels > 1 else np.full(n, 2.0)
    u = rng.uniform(0, 63, n)
    v = rng.uniform(0, 63, n)
    means = np.stack([(u - cx) / f * z, (v - cx) / f * z, z], 1)
    g = dict(means=means.astype(np.float32), log_scales=np.log(1.5 * z / f)[:, None].repeat(3, 1).astype(np.float32),
             quats=np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
             logit_opacity=np.zeros(n, np.float32), sh=np.zeros((n, 1, 3), np.float32))
    return g, cams


@pytest.mark.parametrize("per_tile", [5, 300, 3000])
def test_bucketed_sort_equal_depths(per_tile):
    """Every Gaussian at the same depth: each list is one run of equal keys, ordered by record index (short
    lists: in place, or passes over (depth, record index) when the run is long; long lists: heapsort of the
    run)."""
    g, cams = _level_scene(per_tile, 1, per_tile)
    a, b, c = _all(g, cams, 0)
    _same(a, b, c)
    for t in range(a["ranges"].shape[0]):
        s, e = a["ranges"][t]
        assert np.all(np.diff(a["vals"][s:e]) > 0)  # one depth: index order
    if per_tile == 3000:
        assert (a["ranges"][:, 1] - a["ranges"][:, 0]).max() > 4096


def test_bucketed_sort_depth_levels():
    """Long lists made of runs of equal depth of ~40 to ~100 entries (120 depth values): runs of up to 64
    ordered in registers, longer ones by heapsort."""
    g, cams = _level_scene(5000, 120, 11)
    a, b, c = _all(g, cams, 0)
    _same(a, b, c)
    assert (a["ranges"][:, 1] - a["ranges"][:, 0]).min() > 4096


def test_bucketed_sort_without_block_masks():
    """No schedule: the sort writes no block masks (and reads no conics); lists as before."""
    g, cams = _level_scene(5000, 120, 12)
    a, b, c = _all(g, cams, 0, masks=False)
    _same(a, b, c, masks=False)
    g, cams = scenes.random_scene(3000, 1, 13, 200, 150)
    a, b, c = _all(g, cams, 1, masks=False)
    _same(a, b, c, masks=False)


def test_bucketed_sort_isosurface_scene():
    """The 2M-Gaussian isosurface scene at 1080p from four views (lists of up to ~50,000 instances)."""
    from paper_2509_12138_gb300 import workload
    dev = torch.device("cuda", 0)
    scene = workload.isosurface_scene(2_000_000, 16, 4, 1920, 1080, sh_degree=3, seed=3, device=dev, spatial=True)
    params = gs.pack_params(scene.init, 3, dev)
    fr = gs.Frame(scene.n, gs.Units.single(scene.n), 1920, 1080, 3, device=dev, max_instances=6 * scene.n,
                  with_backward=False, with_loss=False)
    for v in range(4):
        out = []
        for design in DESIGNS:
            fr.preprocess(params, scene.cam(v))
            fr.sort(design)
            torch.cuda.synchronize()
            I = fr.instances()
            out.append(dict(status=fr.read_status(), I=I, vals=fr.sorted_vals[:I].cpu().numpy(),
                            ranges=fr.ranges.cpu().numpy(), masks=fr.block_masks[:I].cpu().numpy()))
        _same(*out)


def test_sort_capacity_overflow():
    """Capacity 100 for ~1,000 instances: every design flags the overflow, reports 100 instances and keeps
    valid lists (which instances survive differs: the global and bucketed designs keep the first in record
    order, the depth-first design the nearest)."""
    g, cams = scenes.random_scene(2000, 0, 70, 128, 96)
    for o in _all(g, cams, 0, cap=100):
        assert o["status"] & 2
        assert o["I"] == 100
        r = o["ranges"]
        assert np.all(r[:, 1] <= 100) and np.all(r[:, 0] <= r[:, 1])
        for t in range(r.shape[0]):
            s, e = r[t]
            assert len(set(o["vals"][s:e].tolist())) == e - s


@pytest.mark.parametrize("W,H,views", [(3840, 2160, 2), (2560, 1440, 8), (1920, 1080, 1)])
def test_sort_unit_tile_bits(W, H, views):
    """(unit | tile) ids of 16 bits (two 4K views: both 8-bit instance passes full), of 17 bits (eight 1440p
    views: the depth-first design hands over to the global sort) and of 13 bits (one 1080p view)."""
    g = synth.random_gaussians(3000, 0, 17, extent=0.8, log_scale_range=(-4.0, -2.5))
    cams = synth.orbital_cameras(views, 3.0, width=W, height=H)
    a, b, c = _all(g, cams, 0)
    _same(a, b, c)


@pytest.mark.parametrize("z_far", [1.9, 1e6])
def test_depth_first_sort_depth_range(z_far):
    """Depths log-uniform from 0.5 to z_far: the depth-first design sorts depth keys relative to the nearest
    depth in four 8-bit passes, the top one skipped on the device when every relative key is below 2^24
    (z_far = 1.9: depths within a factor of 4) and run otherwise (z_far = 1e6).  Lists equal the other
    designs' either way."""
    rng = np.random.default_rng(int(z_far) % 97)
    W = H = 128
    cams = scenes.identity_camera(W, H)
    f, cx = float(cams.fx[0]), float(cams.cx[0])
    n = 6000
    z = np.exp(rng.uniform(np.log(0.5), np.log(z_far), n))
    u, v = rng.uniform(0, W - 1, n), rng.uniform(0, H - 1, n)
    means = np.stack([(u - cx) / f * z, (v - cx) / f * z, z], 1)
    g = dict(means=means.astype(np.float32),
             log_scales=np.log(rng.uniform(1.0, 12.0, n) * z / f)[:, None].repeat(3, 1).astype(np.float32),
             quats=np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
             logit_opacity=np.zeros(n, np.float32), sh=np.zeros((n, 1, 3), np.float32))
    a, b, c = _all(g, cams, 0)
    _same(a, b, c)
    fr = gs.Frame(n, gs.Units.single(n), W, H, 0, with_backward=False, with_loss=False)
    fr.preprocess(gs.pack_params(g, 0), gs.pack_cameras(cams))
    torch.cuda.synchronize()
    d = fr.depth.cpu().numpy()[fr.radius.cpu().numpy() > 0].view(np.uint32).astype(np.int64)
    span = int(d.max() - d.min())
    assert (span >= 1 << 24) == (z_far > 2.0), span
