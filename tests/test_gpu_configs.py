"""Parity at the full sizes of the benchmark workloads (ifgf_inputs.WORKLOADS), in the
launch configuration bench.py times (CUDA-graph replay; batched plans autotuned), on
outputs the oracle computes one by one:

  * sphere_4lambda (N = 24,576, FP64): bit-exact tree and relevant cones against the
    oracle plan; every output against the oracle's serial IFGF (1e-10) and against the
    full FP64 direct sum (1e-3 relative l2).
  * sphere_32lambda (N = 393,216, FP64): bit-exact tree and cones; 2,000 sampled
    targets against the direct sum and 2,000 sampled sources of the adjoint against
    the direct adjoint (1e-3); the autograd gradient of ||u||^2 against central
    differences on 64 sampled entries (the loss is quadratic, so differences are
    exact up to rounding).
  * prolate_128lambda (N = 3,145,728, mixed): 4,096 sampled targets against the direct
    sum (1e-3) and the whole field against the FP64 GPU IFGF on the same inputs
    (2e-5: FP32 values and accumulation).
  * cubes_64rhs (N = 1,572,864, 64 plane-wave right-hand sides, tensor cores): 2,048
    sampled targets per right-hand side against the direct sum (1e-3).
  * prolate_128lambda_adaptive (the same spheroid on an adaptive octree, mixed): 4,096
    sampled targets against the direct sum (1e-3), the adjoint on 256 sampled sources
    against the direct adjoint (1e-3), and the adjoint identity on the GPU operator.
  * sphere_256lambda (N = 25,165,824, 8 right-hand sides, mixed; two-level buffers and
    right-hand-side chunks): 1,024 sampled targets per right-hand side against the
    direct sum (1e-3); 256 sampled sources of the adjoint per right-hand side against
    the direct adjoint (1e-3); the adjoint identity <v, A s> = <A^H v, s> on the GPU
    operator (1e-5: FP32 accumulation).
"""
import numpy as np
import pytest

import ifgf_inputs as wi
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_02857_gb300 as pkg
    return torch, pkg


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _plan(pkg, torch, wl, precision, **kw):
    g = pkg.Plan(torch.from_numpy(wl.points()).cuda(), wl.kappa, wl.levels, wl.p_radial, wl.p_angular,
                 wl.leaf_ns, wl.leaf_nc, precision=precision, leaf_max=wl.leaf_max, **kw)
    if precision == "batched":
        g.autotune(wl.nrhs)
    g.set_graphs(True)
    return g


def _tree_bit_exact(g, o, D):
    assert np.array_equal(g.perm(), o.perm())
    for d in range(1, D + 1):
        gk, gs = g.boxes(d)
        ok, os_ = o.boxes(d)
        assert np.array_equal(gk, ok) and np.array_equal(gs, os_), d
    for d in range(3, D + 1):
        ga, gc = g.active(d)
        oa, oc = o.active(d)
        assert np.array_equal(ga, oa) and np.array_equal(gc, oc), d


def test_sphere_4lambda_full(env):
    torch, pkg = env
    wl = wi.WORKLOADS["sphere_4lambda"]
    pts, sig = wl.points(), wl.densities()
    g = _plan(pkg, torch, wl, "fp64")
    o = oracle.Plan(pts, wl.kappa, wl.levels, 3, 5, wl.leaf_ns, wl.leaf_nc)
    _tree_bit_exact(g, o, wl.levels)
    u = g.apply(torch.from_numpy(sig).cuda()).cpu().numpy()
    assert np.max(np.abs(u - o.apply(sig))) < 1e-10 * np.max(np.abs(u))
    ex = oracle.direct(pts, wl.kappa, sig)
    assert rel(u, ex) < 1e-3
    assert g.check() == 0


def test_sphere_32lambda_sampled_forward_adjoint_and_gradient(env):
    torch, pkg = env
    wl = wi.WORKLOADS["sphere_32lambda"]
    pts, sig = wl.points(), wl.densities()
    g = _plan(pkg, torch, wl, "fp64")
    o = oracle.Plan(pts, wl.kappa, wl.levels, 3, 5, wl.leaf_ns, wl.leaf_nc)
    _tree_bit_exact(g, o, wl.levels)
    del o
    tg = wl.target_indices()
    s = torch.from_numpy(sig).cuda()
    u = g.apply(s).cpu().numpy()
    assert rel(u[:, tg], oracle.direct(pts, wl.kappa, sig, tg)) < 1e-3
    v = wi.complex_normal(wl.seed + 400, (1, wl.n))
    w = g.apply_adjoint(torch.from_numpy(v).cuda()).cpu().numpy()
    assert rel(w[:, tg], oracle.direct_adjoint(pts, wl.kappa, v, tg)) < 1e-3
    # gradient of L = ||A sigma||^2 through the autograd binding vs central differences
    x = s[0].clone().requires_grad_(True)
    loss = (pkg.ifgf_apply_autograd(x[None, :], g).abs() ** 2).sum()
    loss.backward()
    grad = x.grad.cpu().numpy()

    def L(y):
        return float((np.abs(g.apply(torch.from_numpy(y[None, :]).cuda()).cpu().numpy()) ** 2).sum())

    h = 1e-2
    base = sig[0].copy()
    for m in wi.sample_targets(wl.n, 64, wl.seed + 300):
        for unit, an in ((1.0, grad[m].real), (1j, grad[m].imag)):
            xp = base.copy(); xp[m] += h * unit
            xm = base.copy(); xm[m] -= h * unit
            fd = (L(xp) - L(xm)) / (2 * h)
            assert abs(fd - an) <= 1e-6 * abs(loss.item()) / wl.n ** 0.5 + 1e-6 * abs(an), (m, fd, an)
    assert g.check() == 0


def test_prolate_128lambda_mixed_sampled_and_vs_fp64_gpu(env):
    torch, pkg = env
    wl = wi.WORKLOADS["prolate_128lambda"]
    pts, sig = wl.points(), wl.densities()
    gm = _plan(pkg, torch, wl, "mixed")
    s = torch.from_numpy(sig).cuda()
    um = gm.apply(s.to(torch.complex64)).cpu().numpy().astype(np.complex128)
    assert gm.check() == 0
    del gm
    g64 = _plan(pkg, torch, wl, "fp64")
    u64 = g64.apply(s).cpu().numpy()
    assert g64.check() == 0
    del g64
    assert rel(um, u64) < 2e-5
    tg = wl.target_indices()
    ex = oracle.direct(pts, wl.kappa, sig, tg)
    assert rel(um[:, tg], ex) < 1e-3
    assert rel(u64[:, tg], ex) < 1e-3


def test_cubes_64rhs_batched_sampled(env):
    torch, pkg = env
    wl = wi.WORKLOADS["cubes_64rhs"]
    pts, sig = wl.points(), wl.densities()
    g = _plan(pkg, torch, wl, "batched", max_nrhs=wl.nrhs)
    u = g.apply(torch.from_numpy(sig.astype(np.complex64)).cuda()).cpu().numpy()
    assert g.check() == 0
    tg = wl.target_indices()
    ex = oracle.direct(pts, wl.kappa, sig, tg)
    for r in range(wl.nrhs):
        assert rel(u[r, tg], ex[r]) < 1e-3, r


def test_sphere_256lambda_mixed_sampled_forward_adjoint(env):
    torch, pkg = env
    wl = wi.WORKLOADS["sphere_256lambda"]
    pts, sig = wl.points(), wl.densities()
    g = _plan(pkg, torch, wl, "mixed", max_nrhs=wl.nrhs)
    st = g.stats()
    assert st["pingpong"] == 1 and st["rhs_chunk"] < wl.nrhs  # the memory-bounded form
    s = torch.from_numpy(sig.astype(np.complex64)).cuda()
    u = g.apply(s).cpu().numpy()
    assert g.check() == 0
    v = wi.complex_normal(wl.seed + 400, (wl.nrhs, wl.n)).astype(np.complex64)
    w = g.apply_adjoint(torch.from_numpy(v).cuda()).cpu().numpy()
    assert g.check() == 0
    # the identity holds for the approximate operator itself (its adjoint is exact)
    lhs = np.vdot(v.astype(np.complex128), u.astype(np.complex128))
    rhs = np.vdot(w.astype(np.complex128), sig)
    assert abs(lhs - rhs) < 1e-5 * abs(lhs), abs(lhs - rhs) / abs(lhs)
    del g
    tg = wl.target_indices()
    ex = oracle.direct(pts, wl.kappa, sig, tg)
    for r in range(wl.nrhs):
        assert rel(u[r, tg], ex[r]) < 1e-3, (r, rel(u[r, tg], ex[r]))
    src = tg[:256]
    exa = oracle.direct_adjoint(pts, wl.kappa, v.astype(np.complex128), src)
    for r in range(wl.nrhs):
        assert rel(w[r, src], exa[r]) < 1e-3, (r, rel(w[r, src], exa[r]))


def test_prolate_128lambda_adaptive_sampled(env):
    torch, pkg = env
    wl = wi.WORKLOADS["prolate_128lambda_adaptive"]
    pts, sig = wl.points(), wl.densities()
    g = _plan(pkg, torch, wl, "mixed")
    st = g.stats()
    assert st["adaptive"] == 1
    s = torch.from_numpy(sig.astype(np.complex64)).cuda()
    u = g.apply(s).cpu().numpy()
    v = wi.complex_normal(wl.seed + 400, (1, wl.n)).astype(np.complex64)
    w = g.apply_adjoint(torch.from_numpy(v).cuda()).cpu().numpy()
    assert g.check() == 0
    lhs = np.vdot(v.astype(np.complex128), u.astype(np.complex128))
    rhs = np.vdot(w.astype(np.complex128), sig)
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)
    del g
    tg = wl.target_indices()
    assert rel(u[:, tg], oracle.direct(pts, wl.kappa, sig, tg)) < 1e-3
    src = tg[:256]
    assert rel(w[:, src], oracle.direct_adjoint(pts, wl.kappa, v.astype(np.complex128), src)) < 1e-3
