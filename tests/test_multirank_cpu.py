"""Host logic of the N > 1 bench path on CPU: two gloo ranks (world size 2).

The path does not shard (each rank advances an independent replica), so the
only cross-rank step is the max-over-ranks reduction of the timed region; these
tests run it with the gloo backend on 127.0.0.1 and check the replica seeds and
the whole-job value.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, w = bench.dist_env()
        local_ms = 10.0 + 5.0 * rank            # rank 1 is the slowest
        t_max = bench.max_over_ranks(local_ms, dist, "cpu")
        wl = synth.PRECISION
        seed = bench.replica_seed(wl.seed, rank)
        pos = synth.uniform_positions(64, wl.L, seed)
        out.put((rank, r, lr, w, t_max, bench.whole_job_value(wl.n, w, 4, t_max), seed, float(pos.sum())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_replica_seeds():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    import synth
    wl = synth.PRECISION
    for rank, r, lr, w, t_max, value, seed, psum in res:
        assert (r, lr, w) == (rank, rank, 2)
        assert t_max == 15.0                           # the max over ranks, on every rank
        assert value == pytest.approx(wl.n * 2 * 4 / 15e-3)
    assert res[0][6] != res[1][6]                      # independent replicas
    assert res[0][7] != res[1][7]


def test_single_rank_defaults():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_value(100, 1, 10, 1000.0) == pytest.approx(1000.0)
    assert bench.replica_seed(7, 0) == 7
    assert np.isfinite(bench.whole_job_value(262144, 8, 10, 20.0))
