#!/usr/bin/env python
"""Throughput of the isosurface 3D-GS training step and render on one GB300.

One step = one optimiser step on one 1920x1080 view: projection, binning +
radix sort, forward blend, masked L1 + SSIM loss, backward (blend replay +
projection), Adam; the projection of each step runs inside the previous step's
Adam kernel (gs_project_bwd_adam_next; --separate-preprocess: its own launch).
Metric: train iters/s at 10M Gaussians, 1080p (plus render
Mpix/s).  Inputs are synthetic (see paper_2509_12138_gb300/workload.py) and
resident in HBM; params + Adam state (9.6 GB) and per-view GT are far larger
than L2, so no explicit flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
Multi-GPU: one process per GPU under torchrun; each rank trains an independent
problem (weak scaling), no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # the metric's workload: 10M Gaussians (16-mode interface), SH degree 3, 1080p, 128 orbital views
    "iso10M-1080p": dict(n=10_000_000, modes=16, views=128, W=1920, H=1080),
    # smaller workloads for quick checks
    "iso1M-1080p": dict(n=1_000_000, modes=8, views=64, W=1920, H=1080),
    "iso200k-540p": dict(n=200_000, modes=8, views=16, W=960, H=540),
    # the 10M scene at the square resolutions the paper trains on (1024^2 and 2048^2)
    "iso10M-1024sq": dict(n=10_000_000, modes=16, views=128, W=1024, H=1024),
    "iso10M-2048sq": dict(n=10_000_000, modes=16, views=64, W=2048, H=2048),
    # small device footprint (about 2.5 GB) for Nsight Compute captures of single kernels
    "iso2M-1080p-prof": dict(n=2_000_000, modes=16, views=4, W=1920, H=1080),
    # batched form: 8 x-slabs with 5% ghosts, uneven populations (28M), 16 masked views each, one
    # graph-captured launch chain per step (metric: (partition, view) units per second)
    "batched28M-1080p": dict(n=28_000_000, modes=8, views=16, W=1920, H=1080,
                             slabs=[500_000, 1_500_000, 2_500_000, 3_500_000, 4_000_000, 4_500_000, 5_500_000,
                                    6_000_000]),
    # merged render of 8 ghost-celled partitions, 100M Gaussians (SH3), 3840x2160, render only
    "merge100M-4k": dict(n=100_000_000, modes=32, views=8, W=3840, H=2160),
}
METRIC = "train iters/s & render Mpix/s at 10M Gaussians 1080p; PSNR vs plain form"
LAMBDA_SSIM = 0.2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="iso10M-1080p", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--deterministic", action="store_true",
                    help="accumulate screen-space gradients in fixed point (bitwise reproducible steps)")
    ap.add_argument("--chunk", type=int, default=1024, help="list entries per chunk job of the blend schedule")
    ap.add_argument("--separate-preprocess", action="store_true",
                    help="a1 as its own launch each step instead of fused into the previous step's Adam kernel")
    ap.add_argument("--sort", default="depth_first", choices=["depth_first", "global"],
                    help="a2 design: records sorted by depth, then instances binned (gs_bin_sort), or one radix "
                         "sort of all instance keys (gs_bin_sort_global)")
    ap.add_argument("--sparse-adam", action="store_true",
                    help="Gaussians without gradient in a step keep their parameters and moments")
    ap.add_argument("--random-order", action="store_true",
                    help="keep the sampler's random point order instead of the extraction's Z-order")
    ap.add_argument("--cpu-window", type=int, default=8, help="CPU sample: 1/(w*w) of the view's pixels")
    ap.add_argument("--experiment", default=None, choices=["learned-init", "ghost-ablation", "cpu-oracle"],
                    help="instead of the throughput line: the plain vs batched + learned-init comparison")
    ap.add_argument("--exp-gaussians", type=int, default=1_000_000)
    ap.add_argument("--exp-steps", type=int, default=3000)
    ap.add_argument("--exp-modes", type=int, default=8, help="learned-init: interface modes")
    ap.add_argument("--exp-width", type=int, default=1920)
    ap.add_argument("--exp-height", type=int, default=1080)
    ap.add_argument("--exp-views", type=int, default=64)
    ap.add_argument("--exp-views-per-step", type=int, default=2, help="learned-init: views per batched step")
    ap.add_argument("--exp-fit-points", type=int, default=2_000_000,
                    help="learned-init: the MLP trains on a random subset of this many source points")
    ap.add_argument("--exp-init-scale", type=float, default=1.0,
                    help="ghost-ablation: factor on the plain initialisation's scale")
    ap.add_argument("--exp-lambda-bg", type=float, default=0.1,
                    help="ghost-ablation: weight of the background-opacity penalty of the 'mask=on+bg' variant "
                         "(0: leave the variant out)")
    ap.add_argument("--exp-seam-delta", type=float, default=0.01,
                    help="ghost-ablation: seam band half-width (x distance of the visible surface from a slab edge)")
    ap.add_argument("--exp-learned-lr", type=float, default=1.0,
                    help="learned-init: factor on the scale, opacity and rotation learning rates of the learned form")
    ap.add_argument("--exp-learned-mean-lr", type=float, default=1.0,
                    help="learned-init: factor on the position learning rates of the learned form")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            if self.uuid and self.uuid not in f[1]:
                continue
            rows.append(f)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def device_uuid(dev):
    try:
        import torch
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ---------------------------------------------------------------- CPU baseline (oracle)
def cpu_window_camera(cams, v, frac: int):
    """Camera block of a centred (W/frac x H/frac) window of view v (same intrinsics, shifted principal point)."""
    import oracle
    cam = oracle.camera_block(cams, v).copy()
    W, H = int(cam[22]), int(cam[23])
    w, h = W // frac, H // frac
    x0, y0 = (W - w) // 2, (H - h) // 2
    cam[14] -= x0
    cam[15] -= y0
    cam[22], cam[23] = w, h
    return cam, (x0, y0, w, h)


class CpuSample:
    """A bounded sample of one training iteration for the FP64 oracle.

    Per-Gaussian stages (projection, projection Jacobian, Adam) run on a 1/gfrac
    subset of the Gaussians and are scaled by gfrac; per-pixel stages (blend,
    loss, reverse replay) run on a centred window holding 1/frac^2 of the view's
    pixels, with every Gaussian that reaches the window, and are scaled by frac^2."""

    def __init__(self, scene, frac: int = 8, gfrac: int = 100, view: int = 1):
        import oracle
        oracle.build()
        self.frac, self.gfrac = frac, gfrac
        g64 = {k: np.asarray(v, np.float64) for k, v in scene.init.items()}
        self.cam, (x0, y0, w, h) = cpu_window_camera(scene.cams, view, frac)
        # the window's GT image and mask, rendered by the oracle from the scene's surfels (set-up, not timed)
        from paper_2509_12138_gb300 import workload
        surf = workload.gt_surfels(scene.pts, scene.nrm, scene.colors, scene.spacing)
        s64 = {k: np.asarray(v, np.float64) for k, v in surf.items()}
        ps = oracle.project(s64, self.cam)
        ssel = np.nonzero(ps["tiles"] > 0)[0]
        rg = oracle.render({k: v[ssel] for k, v in s64.items()}, self.cam, np.ones(3))
        self.gt = rg["img"]
        self.mask = ((1.0 - rg["final_T"]) >= 1.0 / 255.0).astype(np.uint8)
        # Gaussians that reach the window (selection is set-up, not timed)
        p = oracle.project(g64, self.cam)
        sel = np.nonzero(p["tiles"] > 0)[0]
        self.win = {k: v[sel] for k, v in g64.items()}
        sub = np.arange(0, scene.n, gfrac)
        self.sub = {k: v[sub] for k, v in g64.items()}
        self.sub_cam = oracle.camera_block(scene.cams, view)
        self.desc = (f"FP64 oracle, 1 training iteration of the {scene.n}-Gaussian scene estimated from: projection, "
                     f"projection Jacobian and Adam on every {gfrac}th Gaussian (x{gfrac}); blend, loss and reverse "
                     f"replay on a centred {w}x{h} window (1/{frac * frac} of the {scene.width}x{scene.height} view, "
                     f"{len(sel)} Gaussians reach it) (x{frac * frac})")
        self.cores = oracle.num_threads()

    def step(self) -> float:
        """Seconds of one full iteration, estimated from the timed sample."""
        import oracle
        bg = np.ones(3)
        t0 = time.perf_counter()
        oracle.project(self.sub, self.sub_cam)
        n = self.sub["means"].shape[0]
        rng = np.random.default_rng(0)
        g2d = dict(dxy=rng.standard_normal((n, 2)), dconic=rng.standard_normal((n, 3)),
                   dopacity=rng.standard_normal(n), drgb=rng.standard_normal((n, 3)))
        grads = oracle.project_backward(self.sub, self.sub_cam, g2d)
        flat = oracle.flatten_params(self.sub)
        oracle.adam(flat, grads, np.zeros_like(flat), np.zeros_like(flat), 1e-3, 0.9, 0.999, 1e-15, 1)
        t_gauss = time.perf_counter() - t0
        t0 = time.perf_counter()
        r = oracle.render(self.win, self.cam, bg)
        _, dimg = oracle.loss(r["img"], self.gt, self.mask, LAMBDA_SSIM)
        oracle.render_backward(self.win, self.cam, bg, dimg)
        t_pix = time.perf_counter() - t0
        return t_gauss * self.gfrac + t_pix * self.frac * self.frac


def cpu_baseline(scene, frac: int):
    cs = CpuSample(scene, frac)
    t = cs.step()
    return {"value": 1.0 / t, "unit": "iters/s", "cores": cs.cores, "kind": "oracle", "sample": cs.desc,
            "seconds_per_iter_est": t}


# ---------------------------------------------------------------- our arm
def kernel_launch_count(frame, lam, fused_pre=False):
    """Kernels libgs launches for one training step (a1-a6) of this frame (the kernel launches ncu lists
    for the timed steps; the 4-byte memsets of the ticket counters are not kernels)."""
    tile_bits = (frame.n_tiles - 1).bit_length()
    unit_bits = (frame.units.n - 1).bit_length()
    key_bits = 32 + tile_bits + unit_bits
    pre = 0 if fused_pre else 1               # k_preprocess (fused into the previous step's Adam kernel)
    if getattr(frame, "sort_design", "depth_first") == "depth_first" and tile_bits + unit_bits <= 16:
        # visibility scan + compaction (3), 4 depth passes of (hist, scan, scatter), instance counts, their
        # block sums' scan and the emission (3), ceil(unit|tile bits / 8) instance passes, k_ranges32
        sort = 3 + 3 * 4 + 3 + 3 * (-(-(tile_bits + unit_bits) // 8)) + 1
    else:
        passes = min(-(-key_bits // 9), -(-key_bits // 8))  # 9-bit digits when they save a pass
        sort = 3 + 1 + 3 * passes + 1         # tiles scan, k_duplicate, (hist, scan, scatter) per pass, k_ranges
    sched = frame.use_masks
    if sched:
        sort += 2 + 1 + 3 + 1                 # tile order, chunk counts, their scan, chunk jobs
    fwd = 3 if sched else 1                   # chunk partials, combine, stop chunks
    loss = 1 + (2 if lam > 0 else 1) + 1      # mask count, SSIM stats + gradient (or L1), final
    bwd = 1
    adam = 2                                  # fused projection backward + Adam, step counter
    return pre + sort + fwd + loss + bwd + adam


def run_ours(args, wl, rank, world):
    import torch
    import paper_2509_12138_gb300 as gs
    from paper_2509_12138_gb300 import workload

    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2509_12138_gb300 import shard
    # weak scaling: every rank trains its own independent scene (no collective on the data path)
    scene = workload.isosurface_scene(wl["n"], wl["modes"], wl["views"], wl["W"], wl["H"], sh_degree=3,
                                      seed=shard.rank_seed(0, rank), device=dev, spatial=not args.random_order)
    N, W, H = scene.n, scene.width, scene.height
    params = gs.pack_params(scene.init, 3, dev)
    frame = gs.Frame(N, gs.Units.single(N), W, H, 3, device=dev, max_instances=6 * N,
                     deterministic=args.deterministic, chunk=args.chunk)
    frame.sort_design = args.sort
    opt = gs.Adam(params, 3, extent=1.0, lr_steps=7000)
    opt.sparse = bool(args.sparse_adam)
    bg = scene.bg
    V = len(scene.cams)

    # stage boundaries for per-kernel timing (events on the launching stream)
    # a1 of step k + 1 runs fused into step k's projection backward + Adam (gs_project_bwd_adam_next): the
    # updated parameters are projected while still on chip; only the first step of a loop preprocesses
    fuse = not args.separate_preprocess

    def step(v, ev=None, pre=True):
        cam = scene.cam(v)
        if ev: ev[0].record()
        if pre or not fuse:
            frame.preprocess(params, cam)
        if ev: ev[1].record()
        frame.sort()
        if ev: ev[2].record()
        frame.render(bg)
        if ev: ev[3].record()
        frame.loss(scene.gt[v:v + 1], scene.mask[v:v + 1], LAMBDA_SSIM)
        if ev: ev[4].record()
        frame.blend_backward(bg)
        if ev: ev[5].record()
        opt.fused_step(frame, cam, next_cams_dev=scene.cam((v + 1) % V) if fuse else None)
        if ev: ev[6].record()

    stages = ["preprocess", "bin_sort", "render_fwd", "loss", "blend_bwd", "project_bwd_adam"]
    for w in range(args.warmup):
        step(w % V, pre=w == 0)
    torch.cuda.synchronize()
    st = frame.read_status()
    if st != 0:
        raise RuntimeError(f"device status {st} after warm-up")
    instances = frame.instances()
    visible = float((frame.radius[: frame.P] > 0).float().mean())  # Gaussians with a projection in this view
    lens = (frame.ranges[:, 1] - frame.ranges[:, 0]).float()
    nz = lens[lens > 0]
    tile_len = {"nonempty_tiles": int(nz.numel()), "mean": round(float(nz.mean()), 1) if nz.numel() else 0,
                "p99": float(torch.quantile(nz, 0.99)) if nz.numel() else 0, "max": int(lens.max())}

    watch = None
    if world > 1:
        import torch.distributed as dist
        # host heartbeat between phases: a peer that failed is named before the next phase's kernels launch
        watch = shard.PeerWatch(dist.distributed_c10d._get_default_store(), rank, world, timeout_s=120.0)

    def barrier(phase=None):
        if world > 1:
            if phase is not None:
                watch.beat(phase)
                watch.check(phase)
            dist.barrier()

    clocks = ClockSampler(device_uuid(dev))
    clocks.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)] for _ in range(args.steps)]
    barrier(1)  # every rank finished its warm-up
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select exactly the timed launches
    t0.record()
    for k in range(args.steps):
        step((args.warmup + k) % V, evs[k], pre=False)
    t1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    ms_total = t0.elapsed_time(t1)
    stage_ms = np.zeros(len(stages))
    for e in evs:
        for s in range(len(stages)):
            stage_ms[s] += e[s].elapsed_time(e[s + 1])
    stage_ms /= args.steps

    # work counters of the timed views (the blend kernels' algorithmic units), outside the timed region
    pairs = []
    for k in range(min(args.steps, 16)):
        frame.forward(params, scene.cam((args.warmup + k) % V), bg)
        pairs.append(frame.blend_pairs())
    pairs_per_step = {key: float(np.mean([p[key] for p in pairs])) for key in pairs[0]}
    # Gaussians whose nine screen-space gradient values are all zero in a view (those a sparse Adam would
    # skip), over timed views, outside the timed region (no parameter update)
    zero_frac = []
    for k in range(min(args.steps, 8)):
        v = (args.warmup + k) % V
        cam = scene.cam(v)
        frame.preprocess(params, cam)
        frame.sort()
        frame.render(bg)
        frame.loss(scene.gt[v:v + 1], scene.mask[v:v + 1], LAMBDA_SSIM)
        frame.blend_backward(bg)
        g = frame.dxy[:N].abs().sum(1) + frame.dco[:N].abs().sum(1) + frame.drgb[:N, :3].abs().sum(1)
        zero_frac.append(float((g == 0).float().mean()))

    # render-only (a1-a3) for Mpix/s, in the faster forward mode over 8 views spread around the orbit (whole-list
    # walks stop early on opaque views; chunk-parallel compositing wins where pixels rarely stop and on the
    # long lists of edge-on views)
    mode_ms = {}
    probe = [(k * V) // 8 for k in range(8)]
    for whole in (False, True):
        frame.walk_whole_lists = whole
        frame.forward(params, scene.cam(0), bg)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for v in probe:
            frame.forward(params, scene.cam(v), bg)
        t1.record()
        torch.cuda.synchronize()
        mode_ms["whole_lists" if whole else "parallel_chunks"] = round(t0.elapsed_time(t1) / len(probe), 3)
    frame.walk_whole_lists = mode_ms["whole_lists"] < mode_ms["parallel_chunks"]
    torch.cuda.synchronize()
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    r0.record()
    for k in range(args.steps):
        frame.forward(params, scene.cam(k % V), bg)
    r1.record()
    torch.cuda.synchronize()
    ms_render = r0.elapsed_time(r1) / args.steps
    render_mode = {"chosen": "whole_lists" if frame.walk_whole_lists else "parallel_chunks", "ms_per_frame": mode_ms}
    frame.walk_whole_lists = False  # the training step below uses the chunk-parallel forward
    clk = clocks.stop()

    # end to end through the public API with host buffers: each step's GT view and mask are copied from
    # pinned host memory (on a copy stream, one step ahead into a double buffer, so the copy of step k+1
    # overlaps step k's kernels), the step runs and its loss is read back
    gt_host = torch.empty((V, 3, H, W), dtype=torch.float32).pin_memory()
    mask_host = torch.empty((V, H, W), dtype=torch.uint8).pin_memory()
    gt_host.copy_(scene.gt)
    mask_host.copy_(scene.mask)
    gt_dev = [torch.empty((1, 3, H, W), dtype=torch.float32, device=dev) for _ in range(2)]
    mask_dev = [torch.empty((1, H, W), dtype=torch.uint8, device=dev) for _ in range(2)]
    loss_host = torch.empty(args.steps, dtype=torch.float32).pin_memory()
    copy_stream = torch.cuda.Stream(device=dev)
    ready = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    main = torch.cuda.current_stream()

    def fetch(k):
        b, v = k % 2, (args.warmup + k) % V  # the same views as the device-timed loop
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(consumed[b])  # step k-2's loss has read buffer b
            gt_dev[b][0].copy_(gt_host[v], non_blocking=True)
            mask_dev[b][0].copy_(mask_host[v], non_blocking=True)
            ready[b].record(copy_stream)

    torch.cuda.synchronize()
    barrier()
    e0 = time.perf_counter()
    fetch(0)
    for k in range(args.steps):
        if k + 1 < args.steps:
            fetch(k + 1)
        b, v = k % 2, (args.warmup + k) % V
        cam = scene.cam(v)
        if k == 0 or not fuse:
            frame.preprocess(params, cam)
        frame.sort()
        frame.render(bg)
        main.wait_event(ready[b])
        frame.loss(gt_dev[b], mask_dev[b], LAMBDA_SSIM)
        consumed[b].record(main)
        frame.blend_backward(bg)
        opt.fused_step(frame, cam, next_cams_dev=scene.cam((v + 1) % V) if fuse else None)
        loss_host[k:k + 1].copy_(frame.loss_val, non_blocking=True)
    torch.cuda.synchronize()
    e_sec = time.perf_counter() - e0
    barrier()
    return dict(scene=scene, frame=frame, ms_total=ms_total, stage_ms=stage_ms, stages=stages, ms_render=ms_render,
                clocks=clk, e2e_sec=e_sec, instances=instances, tile_len=tile_len, pairs=pairs_per_step,
                render_mode=render_mode, visible=visible, zero_grad_frac=float(np.mean(zero_frac)),
                sort_design=args.sort,
                sparse_adam=bool(args.sparse_adam), fused_pre=fuse, h2d=(3 * H * W * 4 + H * W), d2h=4,
                launches=kernel_launch_count(frame, LAMBDA_SSIM, fuse) * args.steps, N=N, W=W, H=H)


# Blend kernels' algorithmic work: FP32 issue slots (one per lane-operation, FMA and MUFU included) per
# (pixel, list entry) pair that a walk skipping the records whose alpha box misses the pixel's 4x4 block must
# evaluate (gs_blend_pairs counts them on the device): the forward each such entry until the pixel stops (~15
# slots: offset, quadratic form, exp, alpha, tests, T and colour updates), the reverse replay each such entry up
# to n_contrib (~50 slots: alpha, T recovery, colour-behind update, 9 gradient terms).  The pairs of the plain
# per-pixel walk (every entry of the tile's list) are reported beside it as the work the block masks avoid.
FWD_SLOTS_PER_PAIR = 15
BWD_SLOTS_PER_PAIR = 50


# DRAM bytes (read + write) per unit of each stage, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum, one pass, every launch of three timed steps) of the 2M-Gaussian 1080p training step
# (iso2M-1080p-prof) with the kernels as they are now and the points in Z-order; the unit is the one the
# stage's algorithmic work counts.  Given only for the stages whose data stream far exceeds L2 at that size
# (so that their traffic grows in proportion to the units), and reported for the 10M workload in Z-order,
# scaled by the units of the bench's own timed views.
# The depth-first sort's working set (the 10M records' depth pairs, 80 MB) stays in L2 at 2M, so its figure
# comes from a one-pass capture of the sort kernels alone (-k) on the 10M workload itself.
TRAFFIC_WORKLOAD = "iso10M-1080p"
TRAFFIC_CAPTURED_ON = "iso2M-1080p-prof"
TRAFFIC_PER_UNIT = {
    "preprocess": ("gaussian", 290.31, TRAFFIC_CAPTURED_ON),
    "bin_sort": ("instance", 114.20, TRAFFIC_WORKLOAD),
    "render_fwd": None,
    "loss": None,
    "blend_bwd": None,
    "project_bwd_adam": ("gaussian", 1451.90, TRAFFIC_CAPTURED_ON),
    # the same kernel with the next step's projection fused in (gs_project_bwd_adam_next)
    "project_bwd_adam_next": ("gaussian", 1512.19, TRAFFIC_CAPTURED_ON),
}


def rooflines(res, workload=None, issue=None, random_order=False):
    """Achieved vs peak for every stage; returns (dominant stage's roofline, all).  issue: measured FP32 / MUFU
    lane-operation rates of this device (peak.issue_rates), the denominator of the issue-bound stages."""
    peaks = {}
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        peaks = json.load(open(p))
    hbm = peaks.get("hbm_gbs")
    src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    sms = 152
    if issue:
        slots = issue["fp32_tops"]
        slots_src = (f"measured: gs_peak_issue FP32 FMA chains on all {issue['sms']} SMs in this run "
                     f"({issue['fp32_tops']:.2f} T lane-ops/s; MUFU ex2 {issue['mufu_tops']:.2f} T/s); "
                     "FLOP-equivalent = one FP32 issue slot")
    else:
        mhz = peaks.get("sm_max_mhz", 2070.0)
        slots = 128 * sms * mhz * 1e6 / 1e12  # FP32 lane issue slots per second (T/s)
        slots_src = (f"derived: 152 SMs x 128 FP32 lanes x {mhz:.0f} MHz (one issue slot per lane per clock; "
                     "FLOP-equivalent = one FP32 issue slot)")
    N, I, pairs = res["N"], res["instances"], res["pairs"]
    tiles = ((res["W"] + 15) // 16) * ((res["H"] + 15) // 16)
    key_bits = 32 + max(1, (tiles - 1).bit_length())
    passes = min(-(-key_bits // 9), -(-key_bits // 8))  # 9-bit digits when they save a pass
    if res.get("sort_design", "global") == "depth_first" and key_bits - 32 <= 16:
        Vv = N * res["visible"]
        tp = -(-(key_bits - 32) // 8)
        # per record: tile counts read twice (8 B); per visible record: depth read for the nearest depth
        # (4 B), depth read and (relative depth, id) written (12 B), 3 depth passes of 4 B histogram read +
        # 8 B read + 8 B written, the histogram of the top byte (4 B; its pass is skipped when the view's
        # relative depths stay below 2^24), count gather (8 B), emission reads (id, xy, conic, radius: 40 B);
        # per instance: (key, id) written (8 B), tp passes of 20 B (the last writes the record ids to the
        # output), the block mask written by the last pass (2 B), the key read for the ranges (4 B)
        sort_bytes = N * 8 + Vv * (4 + 12 + 3 * 20 + 4 + 8 + 40) + I * (8 + tp * 20 + 2 + 4)
    else:
        sort_bytes = N * 8 + I * (12 + passes * 32 + 16)
    work = {
        # 15 parameter planes read (240 B at SH3); xy pair, conic, rgb, depth, radius, tiles written (60 B)
        "preprocess": ("hbm", N * (15 * 16 + 60)),
        "bin_sort": ("hbm", sort_bytes),
        # params, m, v read and written; the gradient stays in registers; screen gradients read
        # screen gradients and radius of every Gaussian; params, m, v read and written for the updated ones
        # (sparse Adam: those with a non-zero gradient)
        "project_bwd_adam": ("hbm", N * (40 + 4) + N * (1.0 - (res.get("zero_grad_frac", 0.0) if res.get("sparse_adam")
                                                               else 0.0)) * 59 * 4 * 6),
        "loss": ("hbm", res["W"] * res["H"] * (3 * 4 * 3 + 1 + 3 * 4 * 6)),
        "render_fwd": ("alu", pairs["fwd_pairs_masked"] * FWD_SLOTS_PER_PAIR),
        "blend_bwd": ("alu", pairs["bwd_pairs_masked"] * BWD_SLOTS_PER_PAIR),
    }
    units = {"gaussian": N, "instance": I, "fwd_pair": pairs["fwd_pairs"], "bwd_pair": pairs["bwd_pairs"],
             "pixel": res["W"] * res["H"]}
    fused = bool(res.get("fused_pre"))
    if fused:
        # the next step's a1 runs inside the Adam kernel: its records (60 B per Gaussian) are written there, the
        # parameters it reads are already on chip, and the preprocess stage is empty
        work["project_bwd_adam"] = ("hbm", work["project_bwd_adam"][1] + N * 60)
        work.pop("preprocess")
    kernel = {"preprocess": "k_preprocess", "bin_sort": "sort chain",
              "project_bwd_adam": "k_project_bwd_adam1 (+ the next step's a1)" if fused else "k_project_bwd_adam1",
              "loss": "loss kernels", "render_fwd": "k_render_fwd_m + k_render_fwd_combine + k_render_fwd_stop",
              "blend_bwd": "k_render_bwd_m"}
    out = {}
    for name, ms in zip(res["stages"], res["stage_ms"]):
        if name not in work:
            continue
        bound, amount = work[name]
        traffic = None
        # (the captured traffic is that of the dense update)
        tkey = "project_bwd_adam_next" if (fused and name == "project_bwd_adam") else name
        sparse_upd = name == "project_bwd_adam" and res.get("sparse_adam")
        # (the sort's figure is that of the depth-first design)
        other_sort = name == "bin_sort" and res.get("sort_design", "global") != "depth_first"
        if (workload == TRAFFIC_WORKLOAD and not random_order and TRAFFIC_PER_UNIT[tkey] and not sparse_upd
                and not other_sort):
            u, per, _ = TRAFFIC_PER_UNIT[tkey]
            traffic = round(per * units[u])
        if bound == "hbm":
            ach = amount / (ms * 1e-3) / 1e9
            out[name] = {"kernel": kernel[name], "bound": "hbm", "achieved": round(ach, 1), "peak": hbm,
                         "unit": "GB/s", "frac": round(ach / hbm, 4), "traffic": traffic,
                         "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"}
        else:
            ach = amount / (ms * 1e-3) / 1e12
            fwd = name == "render_fwd"
            n_pairs = pairs["fwd_pairs_masked"] if fwd else pairs["bwd_pairs_masked"]
            n_plain = pairs["fwd_pairs"] if fwd else pairs["bwd_pairs"]
            out[name] = {"kernel": kernel[name], "bound": "alu", "achieved": round(ach, 3),
                         "peak": round(slots, 2), "unit": "TFLOP/s",
                         "frac": round(ach / slots, 4), "traffic": traffic, "peak_source": slots_src,
                         "work": f"{n_pairs:.3e} (pixel, list entry) pairs inside the block masks x "
                                 f"{FWD_SLOTS_PER_PAIR if fwd else BWD_SLOTS_PER_PAIR} FP32 issue slots",
                         "work_avoided": f"{n_plain - n_pairs:.3e} pairs of the plain per-pixel walk "
                                         f"({n_plain:.3e}) fall outside the masks"}
        if traffic is not None:
            on = TRAFFIC_PER_UNIT[tkey][2]
            out[name]["traffic_source"] = (f"ncu dram__bytes_read.sum + dram__bytes_write.sum on {on}, "
                                           + (f"scaled to {TRAFFIC_WORKLOAD} by units: " if on != TRAFFIC_WORKLOAD
                                              else "per unit times the units of the timed views: ") +
                                           f"{TRAFFIC_PER_UNIT[tkey][1]} B per {TRAFFIC_PER_UNIT[tkey][0]} x "
                                           f"{units[TRAFFIC_PER_UNIT[tkey][0]]:.4g} {TRAFFIC_PER_UNIT[tkey][0]}s")
        out[name]["share"] = round(float(ms / res["stage_ms"].sum()), 4)
    dom = max(out, key=lambda k: out[k]["share"])
    return out[dom], out


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    config = {"workload": args.workload, "gaussians": wl["n"], "width": wl["W"], "height": wl["H"],
              "views": wl["views"], "sh_degree": 3, "loss": f"masked L1 + {LAMBDA_SSIM} D-SSIM",
              "gradient_accumulation": "int64 fixed point" if args.deterministic else "float atomics",
              "l2": "inputs larger than L2 (params+Adam state 9.6 GB at 10M)",
              "point_order": "random" if args.random_order else "z-order", "chunk": args.chunk,
              "adam": "sparse" if args.sparse_adam else "dense", "sort": args.sort}
    if args.impl == "reference":
        return run_reference(args, wl, rank, world, config)
    if args.experiment == "learned-init":
        return run_learned_init_experiment(args)
    if args.experiment == "ghost-ablation":
        return run_ghost_ablation(args)
    if args.experiment == "cpu-oracle":
        return run_cpu_oracle_timing(args)
    if args.workload.startswith("batched"):
        return run_batched(args, wl)
    if args.workload.startswith("merge"):
        return run_merge(args, wl)
    import torch
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    if world > 1:
        from paper_2509_12138_gb300 import shard as _shard
        # a rank that dies ends the others' next collective after 5 minutes at most instead of a hang
        _shard.init_group("nccl", timeout_s=300.0, device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_12138_gb300 import peak
    issue = peak.issue_rates()  # the issue-bound stages' denominator, measured before the timed region
    res = run_ours(args, wl, rank, world)
    ms_step = res["ms_total"] / args.steps
    t_max = res["ms_total"]
    e2e_sec = res["e2e_sec"]
    from paper_2509_12138_gb300 import shard
    t_max, e2e_sec, r_max = shard.reduce_max([t_max, e2e_sec, res["ms_render"]], device="cuda")
    value = shard.job_throughput([args.steps] * world, t_max)
    mpix = shard.job_throughput([res["W"] * res["H"]] * world, r_max) / 1e6
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
        "render_mpix_s": round(mpix, 1), "render_ms": round(res["ms_render"], 4), "render_mode": res["render_mode"],
        "stage_ms": {k: round(float(v), 4) for k, v in zip(res["stages"], res["stage_ms"])},
        "instances_per_view": res["instances"], "tile_list_len": res["tile_len"],
        "visible_fraction": round(res["visible"], 4),
        "zero_gradient_fraction": round(res["zero_grad_frac"], 4),
        "e2e": {"value": round(shard.job_throughput([args.steps] * world, e2e_sec * 1e3), 3), "unit": "iters/s",
                "h2d_bytes_per_step": res["h2d"], "d2h_bytes_per_step": res["d2h"]},
        "gpu_launches": res["launches"], "clocks": res["clocks"],
    }
    line["roofline"], line["stage_rooflines"] = rooflines(res, args.workload, issue, args.random_order)
    line["blend_pairs_per_view"] = {k: round(v) for k, v in res["pairs"].items()}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(res["scene"], args.cpu_window)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_learned_init_experiment(args):
    """Plain form vs batched + learned-init form on a scene the MLP has not seen: held-out PSNR against
    wall-clock time (one JSON line)."""
    import torch
    from paper_2509_12138_gb300 import experiment as X
    from paper_2509_12138_gb300 import workload
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    n, W, H, V, steps = args.exp_gaussians, args.exp_width, args.exp_height, args.exp_views, args.exp_steps
    modes = args.exp_modes
    every = max(steps // 15, 1)
    t_scene = time.perf_counter()
    src = workload.isosurface_scene(n, modes, V, W, H, sh_degree=3, seed=101)
    t_scene = time.perf_counter() - t_scene
    h_src, trained = X.run_plain(src, steps, every)
    t0 = time.perf_counter()
    w, losses = X.fit_mlp(src, trained, steps=600, fit_points=args.exp_fit_points)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    del src, trained
    torch.cuda.empty_cache()
    dst = workload.isosurface_scene(n, modes, V, W, H, sh_degree=3, seed=202)
    h_plain, _ = X.run_plain(dst, steps, every)
    target = h_plain.psnr[-1] - 0.1
    from paper_2509_12138_gb300.raster import LearningRates
    f = args.exp_learned_lr
    d = LearningRates()
    fm = args.exp_learned_mean_lr
    lrs = LearningRates(mean_init=d.mean_init * fm, mean_final=d.mean_final * fm, scale=d.scale * f,
                        opacity=d.opacity * f, rotation=d.rotation * f)
    vps = args.exp_views_per_step
    h_learn, _ = X.run_learned_batched(dst, w, steps, every, views_per_step=vps, lrs=lrs, stop_at=target)
    s_hit, t_hit = h_learn.time_to(target)
    fit = None if t_hit is None else round(t_hit + t_fit, 3)
    fit_src = None if t_hit is None else round(t_hit + t_fit + h_src.seconds[-1], 3)
    line = {"experiment": "learned-init vs plain", "gaussians": n, "modes": modes, "width": W, "height": H,
            "views": V, "scene_build_seconds": round(t_scene, 1),
            "plain": {"steps": steps, "seconds": round(h_plain.seconds[-1], 3), "psnr": round(h_plain.psnr[-1], 3),
                      "psnr_at_init": round(h_plain.psnr[0], 3)},
            "batched_learned": {"views_per_step": vps, "lr_factor_scale_opacity_rotation": f,
                                "lr_factor_position": fm,
                                "psnr_at_init": round(h_learn.psnr[0], 3),
                                "steps_to_plain_psnr_minus_0.1dB": s_hit,
                                "seconds_to_plain_psnr_minus_0.1dB": None if t_hit is None else round(t_hit, 3),
                                "seconds_with_mlp_fit": fit,
                                "seconds_with_mlp_fit_and_source_training": fit_src,
                                "final_psnr": round(h_learn.psnr[-1], 3)},
            "mlp": {"fit_seconds": round(t_fit, 3), "source_training_seconds": round(h_src.seconds[-1], 3),
                    "fit_points": min(args.exp_fit_points, n),
                    "loss_first": losses[0], "loss_last": losses[-1],
                    "trained_on": "converged splats of another seed of the interface"},
            "history": {"plain": [h_plain.steps, [round(x, 3) for x in h_plain.seconds],
                                  [round(x, 3) for x in h_plain.psnr]],
                        "learned": [h_learn.steps, [round(x, 3) for x in h_learn.seconds],
                                    [round(x, 3) for x in h_learn.psnr]]}}
    print(json.dumps(line))
    return 0


def run_ghost_ablation(args):
    """Ghost cells and background masks on / off: PSNR of the merged render on held-out views, over all
    covered pixels and over the seam band around the slab boundaries (one JSON line)."""
    import torch
    from paper_2509_12138_gb300 import experiment as X
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    slabs, W, H, V = [args.exp_gaussians // 4] * 4, 960, 540, 32
    res = X.ghost_ablation(slabs, 8, V, W, H, args.exp_steps, n_parts=4, ghost=0.05, sh_degree=1,
                           delta=args.exp_seam_delta, init_scale=args.exp_init_scale, lambda_bg=args.exp_lambda_bg)
    print(json.dumps({"experiment": "ghost cells x masks", "gaussians": sum(slabs), "partitions": 4, "ghost": 0.05,
                      "width": W, "height": H, "views": V, "steps": args.exp_steps,
                      "init_scale": args.exp_init_scale, "lambda_bg": args.exp_lambda_bg,
                      "seam_band": f"pixels whose surface lies within {args.exp_seam_delta} (x) of an interior slab "
                                   "boundary",
                      "results": res}))
    return 0


def _cpu_model() -> str:
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu model")):
                return ln.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _oracle_iteration(g64, cams, views, gt, mask, lam):
    """One measured FP64 training iteration of the oracle: for each view its render, loss, reverse replay and
    projection Jacobian; then one Adam step over all parameters.  Returns seconds."""
    import oracle
    bg = np.ones(3)
    t0 = time.perf_counter()
    grads = 0.0
    for k, v in enumerate(views):
        cam = oracle.camera_block(cams, v)
        r = oracle.render(g64, cam, bg)
        _, dimg = oracle.loss(r["img"], gt[k], mask[k], lam)
        g2d = oracle.render_backward(g64, cam, bg, dimg)
        grads = grads + oracle.project_backward(g64, cam, g2d)
    flat = oracle.flatten_params(g64)
    oracle.adam(flat, grads, np.zeros_like(flat), np.zeros_like(flat), 1e-3, 0.9, 0.999, 1e-15, 1)
    return time.perf_counter() - t0


def run_cpu_oracle_timing(args):
    """The FP64 oracle, as it stands, timed on this machine's host cores for one full training iteration
    (measured, not sampled): the small configuration (2,000 Gaussians on the unit sphere, SH0, all eight
    128x128 views, masked L1) and a 1M-Gaussian interface (SH3, one 1920x1080 view, masked L1 + 0.2 D-SSIM).
    Targets are the oracle's own renders (untimed set-up).  One JSON line."""
    import oracle
    import synth
    from paper_2509_12138_gb300 import workload
    oracle.build()
    out = {"experiment": "cpu oracle, measured iterations", "cores": oracle.num_threads(),
           "nproc": os.cpu_count(), "cpu": _cpu_model(), "results": []}
    # small configuration
    n = 2000
    pts, _ = synth.sphere_points(n, 0)
    _, dist = oracle.knn(pts.astype(np.float64), 3)
    ls = np.log(np.maximum(dist.mean(axis=1), 1e-7))
    y00 = 0.5 / math.sqrt(math.pi)
    init = dict(means=pts.astype(np.float64), log_scales=np.repeat(ls[:, None], 3, 1),
                quats=np.tile([1.0, 0, 0, 0], (n, 1)), logit_opacity=np.full(n, math.log(0.1 / 0.9)),
                sh=np.zeros((n, 1, 3)))
    pert = synth.target_perturbation(n, 0)
    target = dict(init, means=init["means"] + pert["mean_noise"], log_scales=init["log_scales"] + pert["log_scale_noise"],
                  logit_opacity=np.full(n, math.log(0.8 / 0.2)), sh=((pert["rgb"] - 0.5) / y00)[:, None, :])
    cams = synth.orbital_cameras(8, 3.0, width=128, height=128)
    gt, mask = [], []
    for v in range(8):
        r = oracle.render(target, oracle.camera_block(cams, v), np.ones(3))
        gt.append(r["img"])
        mask.append(((1.0 - r["final_T"]) >= 1.0 / 255.0).astype(np.uint8))
    t = _oracle_iteration(init, cams, list(range(8)), gt, mask, 0.0)
    out["results"].append({"config": "2,000 Gaussians, SH0, 8 views of 128x128, masked L1", "kind": "measured",
                           "seconds_per_iteration": round(t, 3), "iters_per_s": round(1.0 / t, 4)})
    # 1M-Gaussian interface, one 1080p view
    n2, W, H = args.exp_gaussians, 1920, 1080
    pts, nrm, _ = synth.interface_points(n2, 8, 0)
    o = synth.spatial_order(pts)
    pts, nrm = pts[o], nrm[o]
    col = synth.lambert_colors(pts, nrm)
    sp = workload.spacing_estimate(nrm, n2)
    init2 = {k: np.asarray(v, np.float64) for k, v in workload.plain_init(pts, col, math.log(sp), 3).items()}
    surf = {k: np.asarray(v, np.float64) for k, v in workload.gt_surfels(pts, nrm, col, sp).items()}
    cams2 = synth.orbital_cameras(64, 1.5, center=(0.5, 0.5, 0.5), width=W, height=H)
    r = oracle.render(surf, oracle.camera_block(cams2, 1), np.ones(3))
    m2 = ((1.0 - r["final_T"]) >= 1.0 / 255.0).astype(np.uint8)
    t2 = _oracle_iteration(init2, cams2, [1], [r["img"]], [m2], LAMBDA_SSIM)
    out["results"].append({"config": f"{n2:,} Gaussians, SH3, one 1920x1080 view, masked L1 + 0.2 D-SSIM",
                           "kind": "measured", "seconds_per_iteration": round(t2, 3),
                           "iters_per_s": round(1.0 / t2, 5)})
    print(json.dumps(out))
    return 0


def run_batched(args, wl):
    """Batched form: the partitions x views-per-step units as one graph-captured step, autotuned.  Under
    torchrun each rank takes the partitions of the longest-first assignment (shard.assign_units, computed on
    every rank alike) and trains them as its own batched step: no collective on the data path; a barrier
    around the timed steps and the max of the per-rank times, value = the units of all ranks over it."""
    import torch
    import paper_2509_12138_gb300 as gs
    from paper_2509_12138_gb300 import shard, train as T, tune, workload
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        shard.init_group("nccl", timeout_s=300.0, device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    ps = workload.partitioned_scene(wl["slabs"], wl["modes"], wl["views"], wl["W"], wl["H"], n_parts=8, ghost=0.05)
    train_v, test_v = T.split_views(wl["views"], 8)
    mine = shard.assign_units(np.diff(ps.offsets), world)[rank]
    idx, off = shard.partition_subset(ps.offsets, mine)
    if world > 1 and mine:  # this rank's partitions only
        init = gs.pack_params({k: np.asarray(v)[idx] for k, v in ps.init.items()}, 3)
        gt, mask = ps.gt[mine].contiguous(), ps.mask[mine].contiguous()
    elif world > 1:
        init = gt = mask = None
    else:
        init, gt, mask = gs.pack_params(ps.init, 3), ps.gt, ps.mask

    def make(variant, vps, chunk=1024):
        return T.BatchedTrainer(init.clone(), 3, off, ps.cams_dev, gt, mask, train_v,
                                views_per_step=vps, variant=variant, lr_steps=7000, chunk=chunk)

    # a rank without partitions (more ranks than partitions) joins the barriers and reductions with no work
    tr, best, table = None, None, {}
    if mine:
        best, table = tune.autotune(make, f"batched28M-{wl['W']}x{wl['H']}-{len(mine)}parts",
                                    candidates=[(0, 1, 1024), (0, 1, 512), (1, 1, 1024), (0, 2, 1024)],
                                    steps=3, warmup=2, use_cache=False)
        tr = make(*best)
        for _ in range(args.warmup):
            tr.step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps if tr is not None else 0):
        tr.step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_max = shard.reduce_max([ms], device="cuda")[0]
    units = tr.units.n * args.steps if tr is not None else 0
    if dist is not None:
        u = torch.tensor([units], dtype=torch.int64, device="cuda")
        dist.all_reduce(u)
        units = int(u.item())
    sec = t_max / 1e3 / args.steps
    # host time of a step: the graph replay of the one gs_train_batch call (views chosen on the device)
    h0 = time.perf_counter()
    for _ in range(args.steps if tr is not None else 0):
        tr.step()
    host_us = (time.perf_counter() - h0) / args.steps * 1e6
    torch.cuda.synchronize()
    st = tr.check() if tr is not None else 0
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {"metric": "batched train step, 8 ghost-celled partitions (28M Gaussians) x views per step, 1080p",
            "value": round(units / (t_max / 1e3), 3), "unit": "(partition, view) units/s",
            "steps_per_s": round(1.0 / sec, 3), "ms_per_step": round(sec * 1e3, 3),
            "host_us_per_step": round(host_us, 1), "n_gpus": world, "scaling": "strong",
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "config": {"workload": args.workload, "gaussians_with_ghosts": int(ps.offsets[-1]),
                                            "slab_sizes": wl["slabs"], "views_per_partition": wl["views"],
                                            "partitions_of_rank0": mine,
                                            "graph": True, "autotune": {"best": best, "units_per_s": table}},
            "status": st}
    print(json.dumps(line))
    return 0


def run_merge(args, wl):
    """Render-only merged scene: ghost-filtered render of all partitions at 4K."""
    import torch
    import paper_2509_12138_gb300 as gs
    from paper_2509_12138_gb300 import workload
    import synth
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    params, xs = workload.interface_gaussians_device(wl["n"], wl["modes"], seed=0)
    params, off, boxes, closed = workload.partition_device(params, xs, 8, 0.05)
    del xs
    torch.cuda.empty_cache()
    N = params.shape[1]
    owned = gs.Owned(off, boxes, closed)
    cams = synth.orbital_cameras(wl["views"], 1.5, center=(0.5, 0.5, 0.5), width=wl["W"], height=wl["H"])
    camd = gs.pack_cameras(cams)
    fr = gs.Frame(N, gs.Units.single(N), wl["W"], wl["H"], 3, with_backward=False, with_loss=False,
                  max_instances=1 << 20)
    need = max(fr.fit_capacity(params, camd[v * 96:(v + 1) * 96], owned) for v in range(wl["views"]))
    fr.set_capacity(int(need * 1.1) + 4096)
    V = wl["views"]
    # forward mode: whole-list walks (opaque renders stop early) or chunk-parallel compositing, whichever
    # renders the warm-up views faster
    mode_ms = {}
    for whole in (True, False):
        fr.walk_whole_lists = whole
        fr.forward(params, camd[0:96], (1.0, 1.0, 1.0), owned)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for k in range(args.warmup):
            fr.forward(params, camd[(k % V) * 96:(k % V + 1) * 96], (1.0, 1.0, 1.0), owned)
        t1.record()
        torch.cuda.synchronize()
        mode_ms["whole_lists" if whole else "parallel_chunks"] = round(t0.elapsed_time(t1) / max(args.warmup, 1), 3)
    fr.walk_whole_lists = mode_ms["whole_lists"] <= mode_ms["parallel_chunks"]
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for k in range(args.steps):
        v = (args.warmup + k) % V
        cam = camd[v * 96:(v + 1) * 96]
        ev[k][0].record()
        fr.preprocess(params, cam, owned)
        ev[k][1].record()
        fr.sort()
        ev[k][2].record()
        fr.render((1.0, 1.0, 1.0))
        ev[k][3].record()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    stage = {name: round(float(np.mean([e[i].elapsed_time(e[i + 1]) for e in ev])), 3)
             for i, name in enumerate(["preprocess", "bin_sort", "render_fwd"])}
    st = fr.read_status()
    kept = int((fr.radius > 0).sum())
    line = {"metric": "merged render (ghost filter + projection + sort + blend), 100M Gaussians SH3, 3840x2160",
            "value": round(wl["W"] * wl["H"] / (ms * 1e-3) / 1e6, 2), "unit": "Mpix/s", "ms_per_frame": round(ms, 3),
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
            "stage_ms": stage, "forward_mode": {"chosen": "whole_lists" if fr.walk_whole_lists else "parallel_chunks",
                                                "warmup_ms_per_frame": mode_ms},
            "data": "synthetic", "config": {"workload": args.workload, "gaussians_with_ghosts": N,
                                            "partitions": 8, "ghost": 0.05, "visible_after_filter_last_view": kept,
                                            "instances_last_view": fr.instances()},
            "status": st}
    print(json.dumps(line))
    return 0


def run_reference(args, wl, rank, world, config):
    """The oracle, as it stands, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return 0
    import oracle
    from paper_2509_12138_gb300 import workload
    oracle.build()
    # host-only scene: the oracle renders the GT of its own sample window (no device code runs in this arm)
    scene = workload.isosurface_points(wl["n"], wl["modes"], wl["views"], wl["W"], wl["H"], sh_degree=3, seed=0)
    # each step is a bounded sample (~4 s of host work at the default size); long runs take a smaller one so
    # that the whole run stays within a few minutes (the estimate of a full iteration scales with it)
    many = args.steps + args.warmup > 20
    cs = CpuSample(scene, max(args.cpu_window, 12) if many else args.cpu_window, gfrac=250 if many else 100)
    for _ in range(args.warmup):
        cs.step()
    times = [cs.step() for _ in range(args.steps)]
    cb = {"cores": cs.cores, "sample": cs.desc}
    t = float(np.mean(times))
    line = {"metric": METRIC, "impl": "reference", "value": round(1.0 / t, 6), "unit": "iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "cpu_baseline": {"value": round(1.0 / t, 6), "unit": "iters/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": round(1.0 / t, 6), "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
