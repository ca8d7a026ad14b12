"""The N>1 path of the benchmark on CPU: two gloo ranks, one process each
(127.0.0.1 rendezvous).  Each rank works on its own donor repertoire (seeded
by rank, weak scaling, no data-path collective); the whole-job reduction takes
the slowest rank's time and the sum of all ranks' units."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2602_17330_gb300 import synth

        # per-rank work as bench.py does it: the rank's own donor
        rep = synth.donor_repertoire(2_000, seed=rank)
        total_ms = 10.0 + 5.0 * rank  # rank 1 is the slowest
        units = float(1000 * (rank + 1))
        max_ms, all_units = bench.whole_job(total_ms, units, world, "cpu")
        np.save(os.path.join(out_dir, f"rank{rank}.npy"),
                np.array([max_ms, all_units, float(rep.codes[:50].sum())], dtype=np.float64))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_whole_job_reduction(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    # every rank sees the same reduction: slowest time, summed units
    assert r0[0] == r1[0] == 15.0
    assert r0[1] == r1[1] == 3000.0
    # the ranks' donors differ (seeded by rank): no shared data path
    assert r0[2] != r1[2]


def test_single_rank_reduction_is_identity():
    import bench

    assert bench.whole_job(12.5, 7.0, 1, "cpu") == (12.5, 7.0)
