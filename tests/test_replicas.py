"""Host logic of the multi-GPU bench (replicas only: the path does not shard, each rank solves its own
instance): run as two gloo ranks on the CPU, the whole-job time is the slowest rank's, and the ranks
get independent instances of the same recipe."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(10.0 + 5.0 * rank, world, device="cpu")
        out[rank] = t
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert dict(out) == {0: 15.0, 1: 15.0}


def test_single_rank_is_its_own_max():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_replicas_solve_independent_instances():
    import bench
    a, b = bench.replica_problem("cfg1", 0), bench.replica_problem("cfg1", 1)
    assert a.m == b.m and np.array_equal(a.val, b.val)   # fixed named workloads are shared
    p0, p1 = bench.replica_problem("cfg2", 0), bench.replica_problem("cfg2", 1)   # the bench workload
    assert (p0.m, p0.n, p0.nnz) == (p1.m, p1.n, p1.nnz) == (65280, 12800, 14400000)
    assert np.array_equal(p0.row_ptr, p1.row_ptr) and not np.array_equal(p0.k, p1.k)
