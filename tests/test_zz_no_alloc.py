"""ifgf_apply_noalloc through the C ABI: the allocation-free evaluation (all scratch
in the library's fixed 64 MiB device array) must give what ifgf_apply gives.

It is meant for callers that may not allocate device memory while evaluating
(memory owned by a framework pool or a fixed budget).  This file is collected
last so that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import ifgf_inputs as wi

pytestmark = pytest.mark.gpu


def _setup():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_02857_gb300 as pkg
    return torch, pkg


def _call(pkg, plan, sigma, u, nrhs, torch):
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = pkg.lib().ifgf_apply_noalloc(plan.handle, ctypes.c_void_p(sigma.data_ptr()),
                                      ctypes.c_void_p(u.data_ptr()), nrhs, st)
    return rc


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_noalloc_matches_apply_on_two_calls(precision, tol):
    torch, pkg = _setup()
    wl = wi.small_sphere(2400, 3, 4, leaf_ns=2, leaf_nc=4, nrhs=2)
    pts = torch.from_numpy(wl.points()).cuda()
    plan = pkg.Plan(pts, wl.kappa, 4, 3, 5, 2, 4, max_nrhs=2, precision=precision)
    sig = torch.from_numpy(wl.densities()).to(plan.complex_dtype).cuda().contiguous()
    ref = plan.apply(sig).cpu().numpy()
    for call in range(2):
        u = torch.full_like(sig, complex(float("nan"), float("nan")))
        assert _call(pkg, plan, sig, u, 2, torch) == 0
        torch.cuda.synchronize()
        got = u.cpu().numpy()
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err <= tol, (call, err)
    assert plan.check() == 0


def test_noalloc_second_plan_and_scratch_limit():
    torch, pkg = _setup()
    # a different plan after the first: the shared array's old contents must not leak
    wl = wi.small_sphere(1800, 2, 4, nrhs=1)
    plan = pkg.Plan(torch.from_numpy(wl.points()).cuda(), wl.kappa, 4, 3, 5, 1, 2)
    sig = torch.from_numpy(wl.densities()).cuda()
    ref = plan.apply(sig).cpu().numpy()
    for _ in range(2):
        u = torch.zeros_like(sig)
        assert _call(pkg, plan, sig, u, 1, torch) == 0
        assert np.max(np.abs(u.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    # a plan whose scratch exceeds the fixed array is rejected, not overrun
    big = wi.WORKLOADS["sphere_4lambda"]
    plan2 = pkg.Plan(torch.from_numpy(big.points()).cuda(), big.kappa, 4, 3, 5, 2, 4, max_nrhs=8)
    sig2 = torch.from_numpy(wi.complex_normal(3, (8, big.n))).cuda()
    u2 = torch.zeros_like(sig2)
    assert _call(pkg, plan2, sig2, u2, 8, torch) == 1  # IFGF_EINVAL
    assert b"scratch" in pkg.lib().ifgf_last_error(plan2.handle)
