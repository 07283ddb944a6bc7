"""The multi-GPU logic of bench.py on CPU ranks (gloo, world size 2): each rank runs its own
independent problem (its own seed), and the job reports the slowest rank's time with the work
of all ranks (weak scaling, no collective on the data path)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    class A:
        precision, periodic, se_target, paths, max_paths = "kahan", 0, 1e-4, 100000, 1 << 25
        iface_stride, form, tau = 0, 0, 1e-2

    prob = bench.workload(A, rank)
    T, ps, est = bench.reduce_over_ranks(dist, 1.0 + rank, 1000 * (rank + 1), 1521, "cpu")
    out[rank] = (prob.seed, T, ps, est)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_aggregation():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
        res = dict(out)
    seeds = {res[r][0] for r in range(2)}
    assert len(seeds) == 2                      # independent problems per rank
    for r in range(2):
        _, T, ps, est = res[r]
        assert T == 2.0                         # slowest rank's time
        assert ps == 3000.0 and est == 2 * 1521  # work of all ranks
