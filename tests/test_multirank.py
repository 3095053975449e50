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
