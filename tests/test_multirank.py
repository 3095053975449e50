"""The multi-GPU run's host logic, on CPU ranks over gloo (world size 2).

The refinement step shards by submap with no collective on the data path;
what remains between ranks is the timing protocol: a barrier around the
timed region, the slowest rank's time, and the sum of the views all ranks
rendered.  These tests run that protocol in two spawned processes and check
the whole-job throughput and that each rank owns a different submap.
"""
import hashlib
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2604_03092_gb300 import multirank


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    from paper_2604_03092_gb300 import scenes
    ri = multirank.rank_info()
    assert (ri.rank, ri.world, ri.local) == (rank, world, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = scenes.random_scene(n=256, width=32, height=24, seed=multirank.submap_seed_offset(rank),
                                 n_views=2 + rank, with_target=False)
        digest = hashlib.sha256(np.ascontiguousarray(sc.means).tobytes()).hexdigest()
        views = len(sc.views) * 3  # three steps of this rank's views
        elapsed_ms = 100.0 + 50.0 * rank  # the ranks finish at different times
        multirank.barrier()
        mx = multirank.max_over_ranks(elapsed_ms)
        total = multirank.sum_over_ranks(views)
        rate = multirank.whole_job_rate(total, mx)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{mx} {total} {rate} {digest}\n")
        multirank.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_views(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    rows = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(world)]
    for mx, total, rate, _ in rows:
        assert float(mx) == 150.0                      # the slowest rank's time
        assert float(total) == (2 + 3) * 3            # views of both ranks
        assert float(rate) == pytest.approx(15 / 0.150)
    assert rows[0][3] != rows[1][3]                    # independent submaps per rank


def test_single_process_reductions_are_identity():
    assert multirank.max_over_ranks(7.5) == 7.5
    assert multirank.sum_over_ranks(32) == 32.0
    multirank.barrier()
    assert multirank.whole_job_rate(64, 500.0) == pytest.approx(128.0)


def test_rank_info_from_environment():
    assert multirank.rank_info({}) == multirank.RankInfo(0, 1, 0)
    assert multirank.rank_info({"WORLD_SIZE": "4", "RANK": "3", "LOCAL_RANK": "1"}) == multirank.RankInfo(3, 4, 1)
    with pytest.raises(ValueError):
        multirank.rank_info({"WORLD_SIZE": "2", "RANK": "2"})
    with pytest.raises(ValueError):
        multirank.whole_job_rate(10, 0.0)


# --------------------------------------------------------------------------
# the views of one submap split across ranks, surfel gradients all-reduced
# --------------------------------------------------------------------------

def _view_shard_worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2604_03092_gb300 import scenes
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = scenes.random_scene(n=300, width=40, height=30, f=35.0, seed=21, n_views=5, with_target=False)
        cfg = oracle.Config()
        g = None
        poses = {}
        for v in multirank.view_shard(len(sc.views), rank, world):
            p = oracle.preprocess_scene_view(sc, v, cfg)
            up = np.random.default_rng(100 + v).normal(size=(8, 30, 40))
            g = oracle.render_bwd(sc.means, sc.scales, sc.quats, p, up, grads=g)
            poses[v] = g.pose.copy()
            g.pose[:] = 0.0  # per-view pose gradients stay with their view
        class G:  # the rank's surfel gradients as tensors
            pass
        t = G()
        for name, _ in multirank.SURFEL_GRAD_FIELDS:
            setattr(t, name, torch.from_numpy(np.ascontiguousarray(getattr(g, name))))
        multirank.allreduce_surfel_grads(t)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"),
                 **{name: getattr(t, name).numpy() for name, _ in multirank.SURFEL_GRAD_FIELDS},
                 **{f"pose{v}": x for v, x in poses.items()})
    finally:
        dist.destroy_process_group()


def test_view_shards_partition_the_views():
    for n in (1, 5, 32):
        for world in (1, 2, 3, 8):
            shards = [multirank.view_shard(n, r, world) for r in range(world)]
            assert [v for s in shards for v in s] == list(range(n))
            assert max(len(s) for s in shards) - min(len(s) for s in shards) <= 1


def test_two_gloo_ranks_sum_view_sharded_surfel_gradients(tmp_path):
    """Two ranks each take half of a submap's views, compute their views'
    surfel gradients and all-reduce them through the package's exchange: on
    both ranks the result equals the single-rank gradient over all views,
    and each view's pose gradient is the single-rank one of that view."""
    import oracle
    from paper_2604_03092_gb300 import scenes
    world = 2
    mp.start_processes(_view_shard_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    sc = scenes.random_scene(n=300, width=40, height=30, f=35.0, seed=21, n_views=5, with_target=False)
    cfg = oracle.Config()
    ref = None
    ref_pose = {}
    for v in range(len(sc.views)):
        p = oracle.preprocess_scene_view(sc, v, cfg)
        up = np.random.default_rng(100 + v).normal(size=(8, 30, 40))
        ref = oracle.render_bwd(sc.means, sc.scales, sc.quats, p, up, grads=ref)
        ref_pose[v] = ref.pose.copy()
        ref.pose[:] = 0.0
    got = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    # FP64 sums in another order (the oracle accumulates with OpenMP atomics,
    # the exchange adds the two ranks' partial sums): equal to ~1e-13 of the
    # largest term, so the bound is set well above that and far below any
    # missing or doubled view's contribution
    for name, _ in multirank.SURFEL_GRAD_FIELDS:
        want = getattr(ref, name)
        assert np.count_nonzero(want) > 0
        for r in range(world):
            np.testing.assert_allclose(got[r][name], want, rtol=1e-9, atol=1e-11 * np.abs(want).max())
    for r in range(world):
        for v in multirank.view_shard(len(sc.views), r, world):
            np.testing.assert_allclose(got[r][f"pose{v}"], ref_pose[v], rtol=1e-9, atol=1e-11 * np.abs(ref_pose[v]).max())
