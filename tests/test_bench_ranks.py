"""bench.py's multi-rank path on the CPU: under torchrun every rank times its own replica (an
independent problem from its own seed, no collective on the data path), the step time is the
largest over the ranks, and the whole-job value counts the cells of every replica.  Two gloo
ranks stand in for two GPUs."""
import multiprocessing as mp
import os
import socket

import numpy as np

import bench
from paper_0901_1110_gb300 import inputs


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.max_over_ranks(ms[rank], dist, "cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_step_time_is_the_max_over_two_gloo_ranks():
    ms = [120.5, 181.25]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert got == [(0, max(ms)), (1, max(ms))]


def test_single_process_max_is_the_value_itself():
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5


def test_whole_job_throughput_counts_every_replica():
    # 2 replicas of 16^3 cells, 5 steps each, the slowest rank taking 250 ms
    assert np.isclose(bench.replica_throughput(2, 16 ** 3, 5, 250.0), 2 * 16 ** 3 * 5 / 0.25)
    assert np.isclose(bench.replica_throughput(1, 8, 1, 1000.0), 8.0)


def test_replicas_draw_independent_problems():
    """The seed is the rank: the density fields and source lists differ between ranks."""
    w0 = inputs.config_lognormal(16, nsrc=4, seed=0)
    w1 = inputs.config_lognormal(16, nsrc=4, seed=1)
    assert w0.nH.shape == w1.nH.shape
    assert not np.allclose(w0.nH, w1.nH)
    assert not np.array_equal(w0.src_ijk, w1.src_ijk)
