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


def test_node_ranges_partition_the_interface_nodes():
    import bench
    for M in (0, 1, 5, 61, 1521, 2032):
        for world in (1, 2, 3, 8):
            r = bench.node_ranges(M, world)
            assert r[0][0] == 0 and r[-1][1] == M and len(r) == world
            assert all(a[1] == b[0] for a, b in zip(r[:-1], r[1:]))
            sizes = [hi - lo for lo, hi in r]
            assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1


def _split_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np

    import bench
    import workloads as W
    from oracle import mc
    from oracle.layout import interface_nodes
    from oracle.step import monitor_on_mesh
    prob = W.c0_small_fp64().replace(px=3, py=2, paths_per_node=400)
    x, y = W.sine_mode_mesh(prob, amp=0.02)
    om = monitor_on_mesh(prob, x, y, prob.t0, None)
    nodes = interface_nodes(prob.nx, prob.ny, prob.px, prob.py, prob.periodic)
    M = len(nodes)
    lo, hi = bench.node_ranges(M, world)[rank]
    est = np.full((M, 2), np.nan)
    sub = mc._interface_mc_ids(prob, x, y, om, nodes, np.arange(lo, hi, dtype=np.int32), 0, np.float64)
    est[lo:hi] = sub[0]
    full = bench.allgather_node_estimates(dist, est, bench.node_ranges(M, world), rank, "cpu")
    out[rank] = full
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_interface_nodes_and_assemble_the_estimates():
    """The node split of one problem over two ranks: each rank estimates its range of interface
    nodes (here with the oracle), one all-gather assembles them, and every rank holds bitwise the
    estimates of all nodes computed at once (each node's paths carry its own node id)."""
    import numpy as np

    import workloads as W
    from oracle import mc
    from oracle.layout import interface_nodes
    from oracle.step import monitor_on_mesh
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_split_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
        res = dict(out)
    prob = W.c0_small_fp64().replace(px=3, py=2, paths_per_node=400)
    x, y = W.sine_mode_mesh(prob, amp=0.02)
    om = monitor_on_mesh(prob, x, y, prob.t0, None)
    nodes = interface_nodes(prob.nx, prob.ny, prob.px, prob.py, prob.periodic)
    ref = mc.interface_mc(prob, x, y, om, nodes, 0, np.float64)[0]
    for r in range(2):
        assert np.array_equal(res[r], ref)
