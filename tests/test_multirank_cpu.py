"""The N>1 path on CPU: two gloo ranks each simulate their replication range
(with the CPU oracle standing in for the device), combine their statistics
with the collectives the multi-GPU run uses (all-reduce of the station rows
and N_K, all-gather of the replication rows), and every rank's combined
buffer equals a single-process run over all replications, bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2402_13259_gb300 import sharding
from paper_2402_13259_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, R, scaling, out_dir):
    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        run = W.tandem3(R=R)
        ranges = [sharding.replica_range(r, world, R, scaling) for r in range(world)]
        begin, count = ranges[rank]
        res = O.simulate(run.net, 1, run.dt, 1.5, count, run.seed, rep_begin=begin)
        counts = [c for _, c in ranges]
        got = sharding.combine_stats_dist(torch.from_numpy(res["stats"]), run.net.n, counts).numpy()
        total = sum(counts)
        whole = O.simulate(run.net, 1, run.dt, 1.5, total, run.seed, rep_begin=0)["stats"]
        assert np.array_equal(got, whole), f"rank {rank}: combined statistics differ"
        # the host-side combination of the same parts agrees
        if rank == 0:
            parts = [O.simulate(run.net, 1, run.dt, 1.5, c, run.seed, rep_begin=b)["stats"] for b, c in ranges]
            assert np.array_equal(sharding.combine_stats(parts, run.net.n, counts), whole)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("scaling", ["strong", "weak"])
def test_two_rank_replication_split(tmp_path, scaling):
    world, R = 2, 37
    port = _free_port()
    mp.spawn(_rank_main, args=(world, port, R, scaling, str(tmp_path)), nprocs=world, join=True)


def test_replica_range_partition():
    for R in (1, 7, 10000):
        for world in (1, 2, 3, 8):
            rs = [sharding.replica_range(r, world, R, "strong") for r in range(world)]
            assert sum(c for _, c in rs) == R
            assert all(rs[k][0] + rs[k][1] == rs[k + 1][0] for k in range(world - 1))
            ws = [sharding.replica_range(r, world, R, "weak") for r in range(world)]
            assert [b for b, _ in ws] == [r * R for r in range(world)]
