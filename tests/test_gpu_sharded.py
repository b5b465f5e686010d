"""Right-hand sides sharded over ranks, through the C ABI on the GPU.

Two processes (a gloo group on the host, both on cuda:0: their kernels never wait on one
another, and the only collective is the host-side gather after the evaluations) each
build a plan of the same geometry and apply their rows of a batch; the gathered rows
equal one process's apply of the whole batch bit for bit (FP64 plans: every kernel's
sums have a fixed order, independent of the other right-hand sides).
"""
import os
import socket
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, nrhs, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import ifgf_inputs as wi
    import paper_2010_02857_gb300 as pkg
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        wl = wi.small_sphere(4000, 4, 5, nrhs=nrhs)
        plan = pkg.Plan(torch.from_numpy(wl.points()).cuda(), wl.kappa, wl.levels, 3, 5, 1, 2, max_nrhs=nrhs)
        sig = torch.from_numpy(wl.densities()).cuda()
        (r0, r1), u = pkg.apply_rhs_sharded(plan, sig, rank, world)
        (_, _), w = pkg.apply_rhs_sharded(plan, sig, rank, world, adjoint=True)
        torch.cuda.synchronize()
        out[rank] = (pkg.gather_rhs_shards(u.cpu().numpy(), nrhs), pkg.gather_rhs_shards(w.cpu().numpy(), nrhs),
                     plan.check())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("nrhs", [4, 8])
def test_rhs_sharded_apply_equals_single_process(nrhs):
    import torch
    import torch.multiprocessing as mp
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    sys.path.insert(0, ROOT)
    import ifgf_inputs as wi
    import paper_2010_02857_gb300 as pkg
    world = 2
    with mp.get_context("spawn").Manager() as m:  # no fork of a process that may hold a CUDA context
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), nrhs, out), nprocs=world, join=True)
        got = [out[r] for r in range(world)]
    wl = wi.small_sphere(4000, 4, 5, nrhs=nrhs)
    plan = pkg.Plan(torch.from_numpy(wl.points()).cuda(), wl.kappa, wl.levels, 3, 5, 1, 2, max_nrhs=nrhs)
    sig = torch.from_numpy(wl.densities()).cuda()
    u = plan.apply(sig).cpu().numpy()
    w = plan.apply_adjoint(sig).cpu().numpy()
    for gu, gw, errs in got:
        assert errs == 0
        assert np.array_equal(gu, u)
        assert np.max(np.abs(gw - w)) <= 1e-12 * np.max(np.abs(w))
