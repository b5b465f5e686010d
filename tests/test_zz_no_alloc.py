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


@pytest.mark.parametrize("precision,flags,tol", [("fp64", 0, 1e-12), ("mixed", 0, 1e-6),
                                                 ("fp64", 8 | 16, 1e-12), ("mixed", 8 | 16, 1e-6)])
def test_noalloc_matches_apply_on_two_calls(precision, flags, tol):
    # flags 8 | 16: a plan with two alternating level buffers that applies 2 right-hand
    # sides per pass; the allocation-free call runs all 4 in one pass with every level
    # resident in its scratch, and must give the same operator
    torch, pkg = _setup()
    nrhs = 4
    wl = wi.small_sphere(2400, 3, 4, leaf_ns=2, leaf_nc=4, nrhs=nrhs)
    pts = torch.from_numpy(wl.points()).cuda()
    plan = pkg.Plan(pts, wl.kappa, 4, 3, 5, 2, 4, max_nrhs=nrhs, precision=precision, flags=flags)
    if flags:
        assert plan.stats()["pingpong"] == 1 and plan.stats()["rhs_chunk"] == 2
    sig = torch.from_numpy(wl.densities()).to(plan.complex_dtype).cuda().contiguous()
    ref = plan.apply(sig).cpu().numpy()
    for call in range(2):
        u = torch.full_like(sig, complex(float("nan"), float("nan")))
        assert _call(pkg, plan, sig, u, nrhs, torch) == 0
        torch.cuda.synchronize()
        got = u.cpu().numpy()
        for r in range(nrhs):
            err = np.max(np.abs(got[r] - ref[r])) / np.max(np.abs(ref[r]))
            assert err <= tol, (call, r, err)
    assert plan.check() == 0


def test_noalloc_batched_plan_runs_the_mixed_kernels():
    # a tensor-core (batched) plan is evaluated here by the mixed-precision CUDA-core
    # kernels: equal to a mixed plan's ifgf_apply up to FP32 rounding, and to the batched
    # plan's own ifgf_apply up to the BF16 operand rounding of the tensor-core path
    torch, pkg = _setup()
    nrhs = 4
    wl = wi.small_sphere(3000, 4, 4, leaf_ns=2, leaf_nc=4, nrhs=nrhs)
    pts = torch.from_numpy(wl.points()).cuda()
    b = pkg.Plan(pts, wl.kappa, 4, 3, 5, 2, 4, max_nrhs=nrhs, precision="batched")
    m = pkg.Plan(pts, wl.kappa, 4, 3, 5, 2, 4, max_nrhs=nrhs, precision="mixed")
    sig = torch.from_numpy(wl.densities()).to(torch.complex64).cuda().contiguous()
    ref_m = m.apply(sig).cpu().numpy()
    ref_b = b.apply(sig).cpu().numpy()
    for call in range(2):
        u = torch.full_like(sig, complex(float("nan"), float("nan")))
        assert _call(pkg, b, sig, u, nrhs, torch) == 0
        torch.cuda.synchronize()
        got = u.cpu().numpy()
        for r in range(nrhs):
            scale = np.max(np.abs(ref_m[r]))
            assert np.max(np.abs(got[r] - ref_m[r])) <= 1e-5 * scale, (call, r)
            assert np.max(np.abs(got[r] - ref_b[r])) <= 2e-3 * scale, (call, r)
    assert b.check() == 0 and m.check() == 0


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
