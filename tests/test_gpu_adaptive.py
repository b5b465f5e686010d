"""GPU parity of the adaptive octree (reading R13: a box of level >= 3 with at most
leaf_max points is a leaf) against the oracle, through the C ABI.

  * tree: boxes, point ranges, leaves, point leaf levels, cousins, near-field ranges and
    relevant cones bit-exact;
  * FP64: near field (1e-12), far field and full apply (1e-10), adjoint (1e-10), the
    adjoint identity on the GPU operator, and the direct sum (1e-3);
  * mixed: every output within the element-wise FP32 bound of the FP64 oracle, with
    resident and with two alternating level buffers.
"""
import math

import numpy as np
import pytest

import ifgf_inputs as wi
import oracle

pytestmark = pytest.mark.gpu

ELEM_MIXED = 1e-4
CASES = [(6, 30), (7, 40), (6, 100000)]  # (D, leaf_max); the last: every box of level 3 a leaf


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_02857_gb300 as pkg
    return torch, pkg


def maxrel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _case(D, kmax):
    pts = wi.spheroid_points(2000, (0.1, 0.1, 1.0), seed=9)
    return pts, 4 * math.pi, D, kmax


@pytest.mark.parametrize("D,kmax", CASES)
def test_adaptive_tree_bit_exact(env, D, kmax):
    torch, pkg = env
    pts, kappa, D, kmax = _case(D, kmax)
    g = pkg.Plan(torch.from_numpy(pts).cuda(), kappa, D, 3, 5, 1, 2, leaf_max=kmax)
    o = oracle.Plan(pts, kappa, D, 3, 5, 1, 2, leaf_max=kmax)
    assert np.array_equal(g.perm(), o.perm())
    assert np.array_equal(g.point_levels(), o.point_levels())
    assert g.stats()["adaptive"] == 1  # every case has leaves above level D
    for d in range(1, D + 1):
        gk, gs = g.boxes(d)
        ok, os_ = o.boxes(d)
        assert np.array_equal(gk, ok) and np.array_equal(gs, os_), d
        ge, gl = g.box_ends(d)
        oe, ol = o.box_ends(d)
        assert np.array_equal(ge, oe) and np.array_equal(gl, ol), d
    for d in range(3, D + 1):
        gs, gl = g.cousins(d)
        os_, ol = o.cousins(d)
        assert np.array_equal(gs, os_) and np.array_equal(gl, ol), d
        for a, b in zip(g.near(d), o.near(d)):
            assert np.array_equal(a, b), d
        ga, gc = g.active(d)
        oa, oc = o.active(d)
        assert np.array_equal(ga, oa) and np.array_equal(gc, oc), d
    assert g.check() == 0


@pytest.mark.parametrize("D,kmax", CASES)
def test_adaptive_fp64_matches_oracle(env, D, kmax):
    torch, pkg = env
    pts, kappa, D, kmax = _case(D, kmax)
    n = len(pts)
    g = pkg.Plan(torch.from_numpy(pts).cuda(), kappa, D, 3, 5, 1, 2, leaf_max=kmax)
    o = oracle.Plan(pts, kappa, D, 3, 5, 1, 2, leaf_max=kmax)
    sig = wi.complex_normal(31, (1, n))
    v = wi.complex_normal(32, (1, n))
    s = torch.from_numpy(sig).cuda()
    assert maxrel(g.apply_partial(s, 1).cpu().numpy(), o.apply(sig, mode=1)) < 1e-12
    assert maxrel(g.apply_partial(s, 2).cpu().numpy(), o.apply(sig, mode=2)) < 1e-10
    u = g.apply(s).cpu().numpy()
    assert maxrel(u, o.apply(sig)) < 1e-10
    w = g.apply_adjoint(torch.from_numpy(v).cuda()).cpu().numpy()
    assert maxrel(w, o.apply_adjoint(v)) < 1e-10
    assert abs(np.vdot(v, u) - np.vdot(w, sig)) < 1e-12 * abs(np.vdot(v, u))
    ex = oracle.direct(pts, kappa, sig)
    assert np.linalg.norm(u - ex) / np.linalg.norm(ex) < 1e-3
    assert g.check() == 0


@pytest.mark.parametrize("flags", [0, 8 | 16])
def test_adaptive_mixed_elementwise_vs_oracle(env, flags):
    torch, pkg = env
    pts, kappa, D, kmax = _case(6, 30)
    n, nrhs = len(pts), 3
    sig = wi.complex_normal(33, (nrhs, n))
    g = pkg.Plan(torch.from_numpy(pts).cuda(), kappa, D, 3, 5, 1, 2, leaf_max=kmax, precision="mixed",
                 max_nrhs=nrhs, flags=flags)
    o = oracle.Plan(pts, kappa, D, 3, 5, 1, 2, leaf_max=kmax)
    s = torch.from_numpy(sig).cuda()
    u, uo = g.apply(s).cpu().numpy(), o.apply(sig)
    w, wo = g.apply_adjoint(s).cpu().numpy(), o.apply_adjoint(sig)
    for r in range(nrhs):
        assert maxrel(u[r], uo[r]) < ELEM_MIXED, (r, maxrel(u[r], uo[r]))
        assert maxrel(w[r], wo[r]) < ELEM_MIXED, (r, maxrel(w[r], wo[r]))
    assert g.check() == 0


def test_adaptive_rejected_for_batched_plans(env):
    torch, pkg = env
    pts, kappa, D, kmax = _case(6, 30)
    with pytest.raises(pkg.IFGFError):
        pkg.Plan(torch.from_numpy(pts).cuda(), kappa, D, 3, 5, 1, 2, leaf_max=kmax, precision="batched", max_nrhs=2)
