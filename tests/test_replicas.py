"""The multi-GPU form of the bench is replicas only (each rank its own views,
no data exchange): two gloo ranks on CPU check the timing reduction (every
rank gets the slowest rank's time), the whole-job throughput and that the
ranks' camera streams are disjoint."""

import os
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    slowest = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    views = synth.sample_views(bench.replica_seed(rank), 0, 8, 64, 64)
    q.put((rank, slowest, views["eye"].copy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_reduce_time_and_draw_disjoint_views():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    assert not np.allclose(out[0][2], out[1][2])

    sys.path.insert(0, ROOT)
    import bench

    # two replicas of 1 Mpixel per step, 10 steps, slowest rank 2 s: 10 Mpixels/s
    assert bench.whole_job_mpix(2, 1_000_000, 10, 2.0) == 10.0
    assert bench.whole_job_mpix(1, 1_000_000, 10, 2.0) == 5.0
