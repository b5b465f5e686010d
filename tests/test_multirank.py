"""Host logic of bench.py's N > 1 path, on CPU ranks of a gloo process group.

With one GPU per rank, bench.py runs independent replicas (no data-path collective): the
job's time is the slowest rank's, taken with an all-reduce MAX after barriers, and only
rank 0 prints.  The reference arm runs on rank 0 alone; the other ranks exit at once.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        out[rank] = bench.max_over_ranks(values[rank])
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_takes_the_slowest_rank():
    import torch.multiprocessing as mp
    world = 2
    values = [12.5, 40.25]
    with mp.get_context("spawn").Manager() as m:  # no fork of a process that may hold a CUDA context
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), values, out), nprocs=world, join=True)
        assert [out[r] for r in range(world)] == [max(values)] * world


def test_max_over_ranks_without_a_group_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


# ------------------------------------------------------------------------------------
# Right-hand sides sharded over ranks
# ------------------------------------------------------------------------------------

def test_rhs_shard_partitions_the_batch():
    sys.path.insert(0, ROOT)
    import paper_2010_02857_gb300 as pkg
    for nrhs in (0, 1, 3, 8, 13, 64):
        for world in (1, 2, 3, 4, 8):
            parts = [pkg.rhs_shard(nrhs, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == nrhs
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        pkg.rhs_shard(4, 2, 2)


def _shard_rank(rank, world, port, out):
    # each rank applies its rows of the batch on its own operator (here the CPU oracle,
    # which stands in for the rank's GPU plan) and the rows are gathered on the host
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import ifgf_inputs as wi
    import oracle
    import paper_2010_02857_gb300 as pkg
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        wl = wi.small_sphere(1500, 2, 4, nrhs=5)
        plan = oracle.Plan(wl.points(), wl.kappa, wl.levels, 3, 5, 1, 2)
        (r0, r1), rows = pkg.apply_rhs_sharded(plan, wl.densities(), rank, world)
        assert rows.shape == (r1 - r0, wl.n)
        out[rank] = pkg.gather_rhs_shards(rows, 5)
    finally:
        dist.destroy_process_group()


def test_rhs_sharded_apply_gathers_the_single_rank_result():
    import numpy as np
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import ifgf_inputs as wi
    import oracle
    world = 2
    with mp.get_context("spawn").Manager() as m:  # no fork of a process that may hold a CUDA context
        out = m.dict()
        mp.spawn(_shard_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        got = [out[r] for r in range(world)]
    wl = wi.small_sphere(1500, 2, 4, nrhs=5)
    ref = oracle.Plan(wl.points(), wl.kappa, wl.levels, 3, 5, 1, 2).apply(wl.densities())
    for g in got:  # every rank holds the whole batch, equal bit for bit
        assert np.array_equal(g, ref)
