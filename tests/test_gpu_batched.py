"""Partitions, batching, graph capture, autotuning and the merged render on the GPU."""
import numpy as np
import pytest
import torch

import oracle
import paper_2509_12138_gb300 as gs
import synth
from paper_2509_12138_gb300 import train as T
from paper_2509_12138_gb300.partition import owned_mask, slab_partition
from tests import scenes
from tests.gpu_util import exclusion_mask, gauss64

pytestmark = pytest.mark.gpu

BG = np.ones(3)


def _subset(g, idx):
    return {k: np.asarray(v)[idx] for k, v in g.items()}


@pytest.mark.parametrize("use_masks,chunk,whole", [(False, 1024, False), (True, 1024, False), (True, 32, False),
                                                   (True, 32, True)])
def test_merge_render_parity(use_masks, chunk, whole):
    """Ghost-filtered merged render equals the oracle's render of the Gaussians the oracle's filter keeps,
    with and without the blend schedule."""
    n, deg, W, H = 3000, 1, 160, 120
    g = synth.random_gaussians(n, deg, 5, center=(0.5, 0.5, 0.5), extent=0.5, log_scale_range=(-4.0, -2.5))
    part = slab_partition(g["means"], 4, 0.1)
    order = part.order
    gp = _subset(g, order)
    # move the means a little, as training does, so that some ghosts leave / enter their slab
    gp["means"] = gp["means"] + np.random.default_rng(0).normal(0, 0.01, gp["means"].shape).astype(np.float32)
    N = len(order)
    cams = scenes.front_camera(W, H, eye=(0.5, -2.0, 1.5), target=(0.5, 0.5, 0.5))
    owned = gs.Owned(part.offsets, part.boxes, part.closed_hi)
    fr = gs.Frame(N, gs.Units.single(N), W, H, deg, with_backward=False, with_loss=False, chunk=chunk)
    fr.use_masks = use_masks
    fr.walk_whole_lists = whole
    params = gs.pack_params(gp, deg)
    camd = gs.pack_cameras(cams)
    fr.fit_capacity(params, camd, owned)
    fr.merge_render(params, camd, BG, owned)
    torch.cuda.synchronize()
    assert fr.read_status() == 0
    part_of = np.repeat(np.arange(part.n), part.sizes())
    keep = oracle.owned(gp["means"], part_of, part.boxes, part.closed_hi)
    assert np.array_equal(keep, owned_mask(gp["means"], part))
    assert (~keep).sum() > 0
    # culled exactly where the filter drops
    rad = fr.radius.cpu().numpy()
    assert np.all(rad[~keep] == 0)
    sub = _subset(gp, np.nonzero(keep)[0])
    cam = oracle.camera_block(cams, 0)
    o = oracle.render(gauss64(sub), cam, BG)
    op = oracle.project(gauss64(sub), cam)
    xy = fr.xy.cpu().numpy()[keep]
    excl, _, flagged = exclusion_mask(op, xy, rad[keep], fr.tiles.cpu().numpy()[keep], o["margin"], W, H)
    assert flagged and excl.mean() < 0.01
    err = np.abs(fr.img.cpu().numpy()[0] - o["img"]).max(axis=0)
    assert err[~excl].max() <= 1e-4


def _partitioned(seed=0, n=6000, W=96, H=72, n_parts=3, views=6):
    pts, nrm, _ = synth.interface_points(n, 4, seed)
    col = synth.lambert_colors(pts, nrm)
    part = slab_partition(pts, n_parts, 0.1)
    from paper_2509_12138_gb300 import workload
    sp = workload.spacing_estimate(nrm, n)
    init = workload.plain_init(pts[part.order], col[part.order], np.log(2 * sp), 1)
    init["logit_opacity"][:] = 0.5
    cams = synth.orbital_cameras(views, 1.6, center=(0.5, 0.5, 0.5), width=W, height=H)
    s = synth.streams(seed + 7, ["gt", "mask"])
    gt = s["gt"].uniform(0, 1, (n_parts, views, 3, H, W)).astype(np.float32)
    mask = (s["mask"].uniform(0, 1, (n_parts, views, H, W)) > 0.3).astype(np.uint8)
    return init, part, cams, gt, mask


def test_batched_partition_units_parity():
    """One batched step over 3 partitions x 2 views: loss and gradients equal the oracle summed per unit."""
    init, part, cams, gt, mask = _partitioned()
    deg = 1
    params = gs.pack_params(init, deg)
    tr = T.BatchedTrainer(params, deg, part.offsets, gs.pack_cameras(cams), torch.from_numpy(gt).cuda(),
                          torch.from_numpy(mask).cuda(), list(range(6)), views_per_step=2, use_graph=False)
    tr._load(0)
    fr = tr.frame
    fr.preprocess(params, tr.cams_step)
    fr.sort()
    fr.render(tr.bg)
    fr.loss(tr.gt_step, tr.mask_step, 0.2)
    fr.backward(params, tr.cams_step, tr.bg)
    torch.cuda.synchronize()
    assert fr.read_status() == 0
    grads = gs.unpack_grads(fr.grads, deg)
    U = tr.units.n
    ref_loss = 0.0
    ref_grad = np.zeros_like(grads)
    u = 0
    for k in range(part.n):
        s, e = part.offsets[k], part.offsets[k + 1]
        sub = gauss64(_subset(init, np.arange(s, e)))
        for j in range(2):
            v = tr.view_of(0, k, j)
            r = oracle.loss_and_grads(sub, oracle.camera_block(cams, v), BG, gt[k, v].astype(np.float64),
                                      mask[k, v], 0.2)
            ref_loss += r["loss"] / U
            ref_grad[s:e] += r["grads"] / U
            u += 1
    assert float(fr.loss_val.item()) == pytest.approx(ref_loss, rel=1e-4)
    scale = np.abs(ref_grad).max()
    assert np.abs(grads - ref_grad).max() <= 1e-3 * scale


def test_train_batch_abi_matches_oracle_per_unit():
    """gs_train_batch called through the C ABI: the views it gathers on the device for step t, the loss and
    the parameter gradient of one batched step over 3 partitions x 2 views equal the oracle summed per unit,
    and the device step counter advances; a second call gathers the views of step t + 1."""
    import ctypes as C
    from paper_2509_12138_gb300 import _lib
    init, part, cams, gt, mask = _partitioned(seed=3)
    deg = 1
    params = gs.pack_params(init, deg)
    tr = T.BatchedTrainer(params, deg, part.offsets, gs.pack_cameras(cams), torch.from_numpy(gt).cuda(),
                          torch.from_numpy(mask).cuda(), list(range(1, 6)), views_per_step=2, use_graph=False)
    tr.keep_grads = True
    tr._build_desc()
    L = _lib.load()
    p0 = gs.unpack_params(params, deg)
    for t in range(2):
        rc = L.gs_train_batch(C.byref(tr.desc), C.c_void_p(tr.frame.status.data_ptr()),
                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        assert tr.frame.read_status() == 0
        assert int(tr.opt.step_dev.item()) == t + 1
        U = tr.units.n
        grads = gs.unpack_grads(tr.frame.grads, deg)
        ref_loss, ref_grad = 0.0, np.zeros_like(grads)
        for k in range(part.n):
            s_, e_ = part.offsets[k], part.offsets[k + 1]
            sub = gauss64(_subset(p0, np.arange(s_, e_)))
            for j in range(2):
                v = tr.view_of(t, k, j)
                u = k * 2 + j
                # the gathered camera, ground truth and mask are those of view v of partition k
                assert torch.equal(tr.gt_step[u].cpu(), torch.from_numpy(gt[k, v]))
                assert torch.equal(tr.mask_step[u].cpu(), torch.from_numpy(mask[k, v]))
                assert torch.equal(tr.cams_step[u * 96:(u + 1) * 96], tr.cams[v * 96:(v + 1) * 96])
                if t == 0:  # the oracle from the (synthetic) initial parameters
                    r = oracle.loss_and_grads(sub, oracle.camera_block(cams, v), BG, gt[k, v].astype(np.float64),
                                              mask[k, v], 0.2)
                    ref_loss += r["loss"] / U
                    ref_grad[s_:e_] += r["grads"] / U
        if t == 0:
            assert float(tr.frame.loss_val.item()) == pytest.approx(ref_loss, rel=1e-4)
            scale = np.abs(ref_grad).max()
            assert np.abs(grads - ref_grad).max() <= 1e-3 * scale


def test_graph_replay_matches_eager():
    """From identical state, one graph replay computes the same step as the eager launch chain: same
    gradients (up to the order of float atomics), same views, same device step counter.  (Parameters are
    not compared across several steps: Adam with eps = 1e-15 turns near-zero gradients into +-lr steps,
    so atomic-order noise in those is amplified; that is the optimiser's definition, not a graph effect.)"""
    init, part, cams, gt, mask = _partitioned(seed=1)
    deg = 1
    mk = lambda g: T.BatchedTrainer(gs.pack_params(init, deg), deg, part.offsets, gs.pack_cameras(cams),
                                    torch.from_numpy(gt).cuda(), torch.from_numpy(mask).cuda(), list(range(6)),
                                    views_per_step=1, use_graph=g)
    tg, te = mk(True), mk(False)
    tg.keep_grads = te.keep_grads = True
    tg.step()  # eager first step + capture
    te.step()
    for a, b in ((te.params, tg.params), (te.opt.m, tg.opt.m), (te.opt.v, tg.opt.v), (te.opt.step_dev, tg.opt.step_dev)):
        a.copy_(b)
    for _ in range(2):
        tg.step()  # graph replay
        te.step()
        torch.cuda.synchronize()
        ga, gb = te.frame.grads, tg.frame.grads
        scale = float(ga.abs().max())
        assert torch.allclose(ga, gb, rtol=1e-4, atol=1e-6 * scale)
        assert abs(float(te.frame.loss_val) - float(tg.frame.loss_val)) <= 1e-5 * abs(float(te.frame.loss_val))
        te.params.copy_(tg.params)
        te.opt.m.copy_(tg.opt.m)
        te.opt.v.copy_(tg.opt.v)
    assert tg.check() == 0 and te.check() == 0
    assert int(tg.opt.step_dev.item()) == int(te.opt.step_dev.item()) == 3


def test_autotuner_picks_and_caches(tmp_path, monkeypatch):
    from paper_2509_12138_gb300 import tune
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "cache.json"))
    init, part, cams, gt, mask = _partitioned(seed=2)
    deg = 1
    gtd, mkd, camd = torch.from_numpy(gt).cuda(), torch.from_numpy(mask).cuda(), gs.pack_cameras(cams)

    def make(variant, vps, chunk=1024):
        return T.BatchedTrainer(gs.pack_params(init, deg), deg, part.offsets, camd, gtd, mkd, list(range(6)),
                                views_per_step=vps, variant=variant, chunk=chunk)

    cands = [(0, 1, 1024), (1, 1, 1024), (2, 2, 1024), (0, 1, 64)]
    best, table = tune.autotune(make, "test", candidates=cands, steps=2, warmup=1)
    assert best in cands and len(table) == 4 and all(v > 0 for v in table.values())
    best2, _ = tune.autotune(make, "test", candidates=[(0, 1)])  # from the cache
    assert best2 == best


@pytest.mark.parametrize("variant", [1, 2])
def test_blend_variants_identical(variant):
    """The execution-shape variants give bit-identical images and identical screen-space gradients up to
    atomic summation order."""
    n, deg, W, H = 2000, 0, 100, 70
    g, cams = scenes.random_scene(n, deg, 3, W, H)
    params = gs.pack_params(g, deg)
    camd = gs.pack_cameras(cams)
    gt, mask = scenes.random_gt(W, H, 4)
    res = []
    for var in (0, variant):
        fr = gs.Frame(n, gs.Units.single(n), W, H, deg, variant=var)
        fr.fit_capacity(params, camd)
        fr.forward(params, camd, BG)
        fr.loss(torch.from_numpy(gt).cuda()[None], torch.from_numpy(mask).cuda()[None], 0.2)
        fr.backward(params, camd, BG)
        torch.cuda.synchronize()
        res.append((fr.img.clone(), fr.n_contrib.clone(), fr.grads.clone()))
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
    assert torch.allclose(res[0][2], res[1][2], rtol=1e-4, atol=1e-7)


@pytest.mark.parametrize("n_views", [1, 2])
def test_fused_projection_backward_adam_matches_separate(n_views):
    """gs_project_bwd_adam == gs_project_bwd followed by gs_adam_step (same gradient, same update), for
    Gaussians in one unit (streaming kernel) and in several views at once (general kernel)."""
    n, deg, W, H = 3000, 3, 120, 90
    g = synth.random_gaussians(n, deg, 21, extent=0.7, log_scale_range=(-3.5, -2.0))
    cams = synth.orbital_cameras(n_views, 3.0, width=W, height=H)
    camd = gs.pack_cameras(cams)
    gts = np.stack([scenes.random_gt(W, H, 22 + k)[0] for k in range(n_views)])
    masks = np.stack([scenes.random_gt(W, H, 22 + k)[1] for k in range(n_views)])
    out = []
    for fused in (False, True):
        params = gs.pack_params(g, deg)
        fr = gs.Frame(n, gs.Units.single(n, n_views), W, H, deg)
        fr.fit_capacity(params, camd)
        opt = gs.Adam(params, deg, extent=1.5, lr_steps=5)
        for _ in range(3):
            fr.forward(params, camd, BG)
            fr.loss(torch.from_numpy(gts).cuda(), torch.from_numpy(masks).cuda(), 0.2)
            fr.blend_backward(BG)
            if fused:
                opt.fused_step(fr, camd, keep_grads=True)
            else:
                fr.project_backward(params, camd)
                opt.step(fr.grads)
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        out.append((params.clone(), opt.m.clone(), fr.grads.clone()))
        if not fused:
            state = (params.clone(), opt.m.clone(), opt.v.clone(), opt.step_dev.clone())
    # one more step from identical state: same gradient and same update
    (p0, m0, v0, s0) = state
    res = []
    for fused in (False, True):
        params = p0.clone()
        fr = gs.Frame(n, gs.Units.single(n, n_views), W, H, deg)
        fr.fit_capacity(params, camd)
        opt = gs.Adam(params, deg, extent=1.5, lr_steps=5)
        opt.m.copy_(m0); opt.v.copy_(v0); opt.step_dev.copy_(s0)
        fr.forward(params, camd, BG)
        fr.loss(torch.from_numpy(gts).cuda(), torch.from_numpy(masks).cuda(), 0.2)
        fr.blend_backward(BG)
        if fused:
            opt.fused_step(fr, camd, keep_grads=True)
        else:
            fr.project_backward(params, camd)
            opt.step(fr.grads)
        torch.cuda.synchronize()
        res.append((params.clone(), opt.m.clone(), opt.v.clone(), fr.grads.clone()))
    (pa, ma, va, ga), (pb, mb, vb, gb) = res
    sc = float(ga.abs().max())
    assert torch.allclose(ga, gb, rtol=1e-4, atol=1e-6 * sc)
    assert torch.allclose(ma, mb, rtol=1e-4, atol=1e-7 * sc)
    assert torch.allclose(pa, pb, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("chunk,opaque,n,whole", [(32, False, 3000, False), (96, False, 3000, False),
                                                  (1024, False, 3000, False), (32, True, 3000, False),
                                                  (96, True, 3000, False), (32, True, 60000, False),
                                                  (32, True, 3000, True), (1024, False, 3000, True)])
def test_schedule_does_not_change_results(chunk, opaque, n, whole):
    """The blend schedule (heaviest-first order, per-instance block masks, lists composited in parallel
    chunks and combined, stop chunks walked again, backward replayed in chunks from the combined
    checkpoints) only skips and reorders work.  Combining per-chunk (T, C) products changes the rounding
    order only: images agree to float rounding, n_contrib exactly, gradients up to atomic order.  Small
    chunks put many chunks on every list; the opaque scenes make most pixels stop after the first chunk,
    so the stop-chunk walk and the checkpoints after a stop are exercised; the dense scene has lists of
    more than 128 chunks.  With whole-list walks the per-pixel arithmetic is that of the unscheduled
    kernel, so images are bit-identical."""
    deg, W, H = 1, 150, 110
    g, cams = scenes.random_scene(n, deg, 31, W, H)
    if opaque:
        g["logit_opacity"][:] = np.log(0.9 / 0.1)
        g["log_scales"][:] += 0.7
    params = gs.pack_params(g, deg)
    camd = gs.pack_cameras(cams)
    gt, mask = scenes.random_gt(W, H, 32)
    res = []
    for use_sched in (False, True):
        fr = gs.Frame(n, gs.Units.single(n), W, H, deg, chunk=chunk)
        fr.use_masks = use_sched
        fr.walk_whole_lists = whole
        fr.fit_capacity(params, camd)
        fr.forward(params, camd, BG)
        fr.loss(torch.from_numpy(gt).cuda()[None], torch.from_numpy(mask).cuda()[None], 0.2)
        fr.backward(params, camd, BG)
        torch.cuda.synchronize()
        assert fr.read_status() == 0
        res.append((fr.img.clone(), fr.n_contrib.clone(), fr.grads.clone(), fr.dco.clone(), fr.final_T.clone()))
        if use_sched:
            lens = (fr.ranges[:, 1] - fr.ranges[:, 0]).cpu().numpy()
            assert int(fr.job_base[-1].item()) == int(np.sum((lens + chunk - 1) // chunk))
            if chunk == 32:
                assert lens.max() > 4 * chunk  # several chunks per list
            if n > 10000:
                assert lens.max() > 128 * chunk
    a, b = res
    if opaque:
        stopped = a[4] < 1e-3
        assert float(stopped.float().mean()) > 0.2  # the early stop is exercised
        assert float((a[1][stopped] > chunk).float().mean()) > 0.3  # ... often after the first chunk
    assert torch.equal(a[1], b[1])
    if whole:
        assert torch.equal(a[0], b[0]) and torch.equal(a[4], b[4])
    assert torch.allclose(a[0], b[0], rtol=0, atol=1e-5)
    assert torch.allclose(a[4], b[4], rtol=1e-4, atol=1e-7)
    sc = float(a[2].abs().max())
    assert torch.allclose(a[2], b[2], rtol=1e-3, atol=1e-5 * sc)
    assert torch.allclose(a[3], b[3], rtol=1e-3, atol=1e-5 * float(a[3].abs().max()))


@pytest.mark.parametrize("whole", [False, True])
def test_stops_hundreds_of_chunks_deep(whole):
    """Pixels that stop after thousands of list entries (hundreds of 32-entry chunks, stop chunks far
    beyond 127): the chunk-parallel forward finds each pixel's stop chunk and walks it again, and the
    backward replays from the checkpoints; results as without the schedule (tests/scenes.deep_stop_scene)."""
    deg, W, H, chunk = 1, 32, 32, 32
    g, cams = scenes.deep_stop_scene(5, W, H)
    n = g["means"].shape[0]
    params = gs.pack_params(g, deg)
    camd = gs.pack_cameras(cams)
    gt, mask = scenes.random_gt(W, H, 6)
    res = []
    for use_sched in (False, True):
        fr = gs.Frame(n, gs.Units.single(n), W, H, deg, chunk=chunk)
        fr.use_masks = use_sched
        fr.walk_whole_lists = whole
        fr.fit_capacity(params, camd)
        fr.forward(params, camd, BG)
        fr.loss(torch.from_numpy(gt).cuda()[None], torch.from_numpy(mask).cuda()[None], 0.2)
        fr.backward(params, camd, BG)
        torch.cuda.synchronize()
        assert fr.read_status() == 0
        res.append((fr.img.clone(), fr.n_contrib.clone(), fr.grads.clone(), fr.final_T.clone()))
    a, b = res
    deep = (a[3] < 1.2e-4) & (a[1] > 128 * chunk)
    assert int(deep.sum()) > 100  # stop chunks beyond 127
    assert torch.equal(a[1], b[1])
    assert torch.allclose(a[0], b[0], rtol=0, atol=1e-5)
    assert torch.allclose(a[3], b[3], rtol=1e-4, atol=1e-7)
    sc = float(a[2].abs().max())
    assert torch.allclose(a[2], b[2], rtol=1e-3, atol=1e-5 * sc)


def test_train_batch_with_bg_penalty_matches_oracle_per_unit():
    """gs_train_batch with the background-opacity penalty (lambda_bg > 0): the loss and the parameter gradient
    of the first step equal the oracle's masked loss plus penalty, per unit, averaged over the 3 x 2 units."""
    import ctypes as C
    from paper_2509_12138_gb300 import _lib
    init, part, cams, gt, mask = _partitioned(seed=5)
    deg, lam_bg = 1, 0.3
    params = gs.pack_params(init, deg)
    tr = T.BatchedTrainer(params, deg, part.offsets, gs.pack_cameras(cams), torch.from_numpy(gt).cuda(),
                          torch.from_numpy(mask).cuda(), list(range(1, 6)), views_per_step=2, use_graph=False,
                          lambda_bg=lam_bg)
    tr.keep_grads = True
    tr._build_desc()
    L = _lib.load()
    p0 = gs.unpack_params(params, deg)
    rc = L.gs_train_batch(C.byref(tr.desc), C.c_void_p(tr.frame.status.data_ptr()),
                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert tr.frame.read_status() == 0
    U = tr.units.n
    grads = gs.unpack_grads(tr.frame.grads, deg)
    ref_loss, ref_grad, pen = 0.0, np.zeros_like(grads), 0.0
    for k in range(part.n):
        s_, e_ = part.offsets[k], part.offsets[k + 1]
        sub = gauss64(_subset(p0, np.arange(s_, e_)))
        for j in range(2):
            v = tr.view_of(0, k, j)
            cam = oracle.camera_block(cams, v)
            r = oracle.render(sub, cam, BG)
            lv, dimg = oracle.loss(r["img"], gt[k, v].astype(np.float64), mask[k, v], 0.2)
            pv, dT = oracle.bg_penalty(r["final_T"], mask[k, v], lam_bg)
            g2d = oracle.render_backward(sub, cam, BG, dimg, dT)
            ref_loss += (lv + pv) / U
            pen += pv / U
            ref_grad[s_:e_] += oracle.project_backward(sub, cam, g2d) / U
    assert pen > 1e-3 * ref_loss
    assert float(tr.frame.loss_val.item()) == pytest.approx(ref_loss, rel=1e-4)
    assert np.abs(grads - ref_grad).max() <= 1e-3 * np.abs(ref_grad).max()
