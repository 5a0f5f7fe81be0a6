"""The multi-GPU host path on the CPU: two gloo ranks (no GPU).

Covers what runs across processes: every rank derives the same unit assignment without communicating,
the measurement's max-over-ranks timing and whole-job throughput, independent per-rank seeds, and the
merge exchange (owned splats of every rank gathered in rank order to the renderer)."""
import os
import socket
import time

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2509_12138_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, outdir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # 1. the same assignment on every rank, computed locally
        sizes = [500_000, 1_500_000, 2_500_000, 3_500_000, 4_000_000, 4_500_000, 5_500_000, 6_000_000]
        asg = shard.assign_units(sizes, world)
        flat = torch.tensor([u for r in asg for u in r] + [len(r) for r in asg], dtype=torch.int64)
        got = [torch.zeros_like(flat) for _ in range(world)]
        dist.all_gather(got, flat)
        same = all(torch.equal(g, flat) for g in got)
        # 2. timing: each rank's own time; the reduction gives the slowest on every rank
        t_local = 10.0 + 5.0 * rank
        t_max, e_max = shard.reduce_max([t_local, 100.0 - rank])
        # 3. merge exchange: rank r owns the Gaussians of its slab; keep flags select them
        n = 5 + 3 * rank
        params = torch.arange(2 * n * 4, dtype=torch.float32).reshape(2, n, 4) + 1000.0 * rank
        keep = torch.tensor([(i % 2 == 0) or rank == 1 for i in range(n)])
        merged = shard.gather_owned(params, keep, dst=0)
        seed = shard.rank_seed(7, rank)
        np.savez(os.path.join(outdir, f"r{rank}.npz"), same=same, t_max=t_max, e_max=e_max,
                 merged=(merged.numpy() if merged is not None else np.zeros(0)), has=merged is not None, seed=seed,
                 mine=np.asarray(asg[rank]))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def two_ranks(tmp_path_factory):
    out = tmp_path_factory.mktemp("gloo")
    mp.start_processes(_worker, args=(2, _free_port(), str(out)), nprocs=2, join=True, start_method="spawn")
    return [np.load(out / f"r{r}.npz") for r in range(2)]


def test_assignment_identical_on_all_ranks_and_covers_each_unit_once(two_ranks):
    assert all(bool(r["same"]) for r in two_ranks)
    units = sorted(int(u) for r in two_ranks for u in r["mine"])
    assert units == list(range(8))


def test_assignment_balances_by_size():
    sizes = [500_000, 1_500_000, 2_500_000, 3_500_000, 4_000_000, 4_500_000, 5_500_000, 6_000_000]
    for world in (1, 2, 4, 8):
        asg = shard.assign_units(sizes, world)
        loads = [sum(sizes[u] for u in r) for r in asg]
        assert sorted(u for r in asg for u in r) == list(range(8))
        # LPT bound: the heaviest rank exceeds the mean by at most the largest unit
        assert max(loads) <= sum(sizes) / world + max(sizes)
    assert shard.assign_units(sizes, 8) == [[7], [6], [5], [4], [3], [2], [1], [0]]
    with pytest.raises(ValueError):
        shard.assign_units(sizes, 0)


def test_timing_is_the_max_over_ranks(two_ranks):
    for r in two_ranks:
        assert float(r["t_max"]) == 15.0 and float(r["e_max"]) == 100.0
    # whole-job throughput: both ranks' units over the slowest rank's time
    assert shard.job_throughput([50, 50], 15.0) == pytest.approx(100 / 0.015)


def test_ranks_get_independent_seeds(two_ranks):
    assert int(two_ranks[0]["seed"]) != int(two_ranks[1]["seed"])
    assert shard.rank_seed(7, 0) == 7


def test_merge_gathers_owned_splats_in_rank_order(two_ranks):
    assert bool(two_ranks[0]["has"]) and not bool(two_ranks[1]["has"])
    expect = []
    for rank in range(2):
        n = 5 + 3 * rank
        p = np.arange(2 * n * 4, dtype=np.float32).reshape(2, n, 4) + 1000.0 * rank
        keep = np.array([(i % 2 == 0) or rank == 1 for i in range(n)])
        expect.append(p[:, keep])
    np.testing.assert_array_equal(two_ranks[0]["merged"], np.concatenate(expect, axis=1))


def test_partition_subset_covers_each_gaussian_once():
    """The ranks' partition subsets of a partition-major layout: each Gaussian in exactly one rank's
    subset, in partition order, with sub-layout offsets of the partitions' sizes."""
    offsets = np.array([0, 7, 7, 20, 26, 41, 50, 61, 80])
    sizes = np.diff(offsets)
    seen = []
    for world in (1, 2, 3, 8):
        seen = []
        for parts in shard.assign_units(sizes, world):
            idx, sub = shard.partition_subset(offsets, parts)
            assert np.array_equal(np.diff(sub), sizes[parts])
            for j, k in enumerate(parts):
                assert np.array_equal(idx[sub[j]:sub[j + 1]], np.arange(offsets[k], offsets[k + 1]))
            seen.extend(idx.tolist())
        assert sorted(seen) == list(range(80))
    with pytest.raises(ValueError):
        shard.partition_subset(offsets, [8])
    with pytest.raises(ValueError):
        shard.partition_subset(offsets, [1, 1])


def test_single_process_paths_need_no_process_group():
    p = torch.ones((3, 4, 4))
    keep = torch.tensor([True, False, True, True])
    assert shard.gather_owned(p, keep).shape == (3, 3, 4)
    assert shard.reduce_max([1.0, 2.0]) == [1.0, 2.0]


def _failing_worker(rank, world, port, outdir):
    """Rank 1 leaves after step 1 (its host loop ends without reporting step 2, as after an exception that
    its own handler swallowed); rank 0 must learn of it from the heartbeat before its next step, and a
    collective with the departed rank must end in an error rather than hang."""
    shard.init_group("gloo", timeout_s=3.0, init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    store = dist.distributed_c10d._get_default_store()
    watch = shard.PeerWatch(store, rank, world, timeout_s=2.0)
    for step in (1, 2):
        if rank == 1 and step == 2:
            os._exit(0)  # the failure, injected on the host: this rank is gone
        watch.beat(step)
        if rank == 0:
            t0 = time.monotonic()
            try:
                watch.check(step)
                res = "ok"
            except shard.PeerFailure as e:
                res = f"failure: {e}"
            dt = time.monotonic() - t0
            if step == 2:
                t1 = time.monotonic()
                try:
                    shard.reduce_max([1.0])
                    coll = "returned"
                except Exception as e:  # the peer is gone: gloo reports it, or the group times out
                    coll = f"error: {type(e).__name__}"
                np.savez(os.path.join(outdir, "fail.npz"), res=res, dt=dt, coll=coll, dt_coll=time.monotonic() - t1)
                os._exit(0)
            assert res == "ok", res


def test_failed_rank_is_detected_on_the_host_and_collectives_do_not_hang(tmp_path):
    ctx = mp.start_processes(_failing_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=False,
                             start_method="spawn")
    t0 = time.monotonic()
    while True:
        if ctx.join(timeout=1):
            break
        if all(not p.is_alive() for p in ctx.processes) or time.monotonic() - t0 > 60:
            break
    for p in ctx.processes:
        if p.is_alive():
            p.kill()
    r = np.load(tmp_path / "fail.npz")
    assert str(r["res"]).startswith("failure: ranks [1] did not report step 2")
    assert 1.5 < float(r["dt"]) < 10.0
    assert str(r["coll"]).startswith("error") and float(r["dt_coll"]) < 30.0
