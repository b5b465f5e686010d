"""GPU parity against the CPU oracle (through the C ABI).

Tolerances:
  * tree, neighbour, cousin and relevant-cone arrays: bit-exact (integer work);
  * FP64 plans vs the oracle's serial IFGF: 1e-10 relative (max-norm over outputs).
    Both evaluate the same interpolants with the same cone choices; they differ only
    in summation order, FMA contraction and the last bits of libm vs CUDA
    transcendentals: ~1e-16 per operation times a few thousand terms;
  * IFGF vs the direct sum (Eq. field1): 1e-3 relative l2 (the accuracy target);
  * mixed plans (FP32 values, FP64 geometry) vs the FP64 oracle IFGF: 2e-5 relative
    l2: FP32 rounding (6e-8) accumulated over ~10^3 terms per output and per level.
"""
import numpy as np
import pytest

import ifgf_inputs as wi
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    return torch


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_02857_gb300 as p
    return p


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def maxrel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


CASES = [
    # n, wavelengths, D, leaf_ns, leaf_nc
    (2000, 2, 4, 1, 2),
    (3001, 4, 4, 2, 4),
    (4099, 3, 5, 1, 2),
    (2500, 0, 4, 1, 2),   # kappa = 0 (Laplace)
]


def _make(case, nrhs=1):
    n, nl, D, ns, nc = case
    wl = wi.small_sphere(n, nl, D, leaf_ns=ns, leaf_nc=nc, nrhs=nrhs)
    return wl, wl.points(), wl.densities()


@pytest.mark.parametrize("case", CASES)
def test_tree_and_cones_bit_exact(pkg, torch_cuda, case):
    wl, pts, _ = _make(case)
    n, nl, D, ns, nc = case
    g = pkg.Plan(pts, wl.kappa, D, 3, 5, ns, nc)
    o = oracle.Plan(pts, wl.kappa, D, 3, 5, ns, nc)
    H1, corner = g.geometry()
    oH1, ocorner = o.geometry()
    assert H1 == oH1 and np.array_equal(corner, ocorner)
    assert np.array_equal(g.perm(), o.perm())
    for d in range(1, D + 1):
        gk, gs = g.boxes(d)
        ok, os_ = o.boxes(d)
        assert np.array_equal(gk, ok) and np.array_equal(gs, os_), d
    for d in range(3, D + 1):
        gs, gl = g.cousins(d)
        os_, ol = o.cousins(d)
        assert np.array_equal(gs, os_) and np.array_equal(gl, ol), d
        ga, gc = g.active(d)
        oa, oc = o.active(d)
        li, oli = g.level_info(d), o.level_info(d)
        assert (li["ns"], li["nc"]) == (oli["ns"], oli["nc"])
        assert np.array_equal(ga, oa) and np.array_equal(gc, oc), d
    assert g.check() == 0


@pytest.mark.parametrize("case,precision", [((12000, 8, 6, 1, 2), "fp64"), ((12000, 8, 6, 1, 2), "mixed"),
                                            ((16000, 4, 5, 3, 6), "mixed")])
def test_rule_ii_by_cone_id_marks_the_same_cones(pkg, torch_cuda, case, precision):
    # relevance rule (ii) marked once per distinct parent cone id and octant (default,
    # where the ids are few against the parent slots) and node by node (flags bit 12):
    # the same relevant cones on every level, and both equal to the oracle's
    wl, pts, _ = _make(case)
    n, nl, D, ns, nc = case
    a = pkg.Plan(pts, wl.kappa, D, 3, 5, ns, nc, precision=precision)
    b = pkg.Plan(pts, wl.kappa, D, 3, 5, ns, nc, precision=precision, flags=4096)
    o = oracle.Plan(pts, wl.kappa, D, 3, 5, ns, nc)
    sa, sb = a.stats()["level"], b.stats()["level"]
    assert any(lv["act_sets"] for lv in sa) and not any(lv["act_sets"] for lv in sb)
    for d in range(3, D + 1):
        ga, gc = a.active(d)
        ha, hc = b.active(d)
        oa, oc = o.active(d)
        assert np.array_equal(ga, ha) and np.array_equal(gc, hc), d
        assert np.array_equal(ga, oa) and np.array_equal(gc, oc), d
    assert a.check() == 0 and b.check() == 0


@pytest.mark.parametrize("case", CASES)
def test_fp64_apply_matches_oracle_and_direct(pkg, torch_cuda, case):
    torch = torch_cuda
    wl, pts, sigma = _make(case, nrhs=1)
    n, nl, D, ns, nc = case
    g = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, D, 3, 5, ns, nc)
    o = oracle.Plan(pts, wl.kappa, D, 3, 5, ns, nc)
    s = torch.from_numpy(sigma).cuda()
    # stage-wise: near field, far field, and cone values of every level
    un = g.apply_partial(s, 1).cpu().numpy()
    assert maxrel(un, o.apply(sigma, mode=1)) < 1e-12
    uf = g.apply_partial(s, 2).cpu().numpy()
    of = o.apply(sigma, mode=2)
    assert maxrel(uf, of) < 1e-10
    for d in range(3, D + 1):
        assert maxrel(g.values(d), o.F(d)) < 1e-10, d
    u = g.apply(s).cpu().numpy()
    uo = o.apply(sigma)
    assert maxrel(u, uo) < 1e-10
    ex = oracle.direct(pts, wl.kappa, sigma)
    assert rel(u, ex) < 1e-3
    assert g.check() == 0


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_order_4_7_matches_oracle(pkg, torch_cuda, precision, tol):
    # (P_s, P_ang) = (4, 7): 196 interpolation points per cone, 18 Lagrange weights
    torch = torch_cuda
    wl, pts, sigma = _make((3000, 3, 4, 2, 4))
    g = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 4, 4, 7, 2, 4, precision=precision)
    o = oracle.Plan(pts, wl.kappa, 4, 4, 7, 2, 4)
    s = torch.from_numpy(sigma).cuda()
    if precision == "fp64":
        o.apply(sigma, mode=2)
        g.apply_partial(s, 2)
        for d in range(3, 5):
            assert maxrel(g.values(d), o.F(d)) < tol, d
    u = g.apply(s).cpu().numpy()
    uo = o.apply(sigma)
    assert rel(u, uo) < tol
    assert rel(u, oracle.direct(pts, wl.kappa, sigma)) < 1e-3
    v = wi.complex_normal(33, (1, wl.n))
    w = g.apply_adjoint(torch.from_numpy(v).cuda()).cpu().numpy()
    assert rel(w, o.apply_adjoint(v)) < tol
    assert g.check() == 0


@pytest.mark.parametrize("case", CASES[:3])
def test_fp64_adjoint_matches_oracle(pkg, torch_cuda, case):
    torch = torch_cuda
    wl, pts, _ = _make(case)
    n, nl, D, ns, nc = case
    v = wi.complex_normal(31, (1, n))
    s = wi.complex_normal(32, (1, n))
    g = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, D, 3, 5, ns, nc)
    o = oracle.Plan(pts, wl.kappa, D, 3, 5, ns, nc)
    vg = torch.from_numpy(v).cuda()
    for mode in (1, 2):
        assert maxrel(g.apply_partial(vg, mode, adjoint=True).cpu().numpy(),
                      o.apply_adjoint(v, mode=mode)) < 1e-10, mode
    w = g.apply_adjoint(vg).cpu().numpy()
    assert maxrel(w, o.apply_adjoint(v)) < 1e-10
    # dot-product test on the GPU operator itself
    u = g.apply(torch.from_numpy(s).cuda()).cpu().numpy()
    assert abs(np.vdot(v, u) - np.vdot(w, s)) < 1e-12 * abs(np.vdot(v, u))
    assert g.check() == 0


def test_multiple_rhs_and_ragged_chunks(pkg, torch_cuda):
    torch = torch_cuda
    wl, pts, _ = _make((2600, 3, 4, 1, 2))
    o = oracle.Plan(pts, wl.kappa, 4, 3, 5, 1, 2)
    for prec, nrhs, tol in [("fp64", 3, 1e-10), ("fp64", 6, 1e-10), ("mixed", 11, 2e-5)]:
        g = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 4, 3, 5, 1, 2, max_nrhs=16, precision=prec)
        sig = wi.complex_normal(40 + nrhs, (nrhs, wl.n))
        u = g.apply(torch.from_numpy(sig).cuda()).cpu().numpy()
        uo = o.apply(sig)
        for r in range(nrhs):
            assert rel(u[r], uo[r]) < tol, (prec, nrhs, r)
        w = g.apply_adjoint(torch.from_numpy(sig).cuda()).cpu().numpy()
        wo = o.apply_adjoint(sig)
        for r in range(nrhs):
            assert rel(w[r], wo[r]) < tol, (prec, nrhs, r)
        assert g.check() == 0


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("mixed", 1e-5)])
def test_upward_tables_match_on_the_fly_geometry(pkg, torch_cuda, precision, tol):
    torch = torch_cuda
    wl, pts, sigma = _make((6000, 4, 6, 1, 2))
    a = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 6, 3, 5, 1, 2, precision=precision)
    b = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 6, 3, 5, 1, 2, precision=precision, flags=2)
    assert any(lv["table_rows"] > 0 for lv in a.stats()["level"])
    assert all(lv["table_rows"] == 0 for lv in b.stats()["level"])
    s = torch.from_numpy(sigma).cuda()
    ua, ub = a.apply(s).cpu().numpy(), b.apply(s).cpu().numpy()
    assert rel(ua, ub) < tol
    wa, wb = a.apply_adjoint(s).cpu().numpy(), b.apply_adjoint(s).cpu().numpy()
    assert rel(wa, wb) < tol
    o = oracle.Plan(pts, wl.kappa, 6, 3, 5, 1, 2)
    assert rel(ua, o.apply(sigma)) < (1e-10 if precision == "fp64" else 2e-5)
    assert a.check() == 0 and b.check() == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cone_index_fast_path_is_exact_on_cell_boundaries(pkg, torch_cuda, precision):
    # vectors on and next to every kind of cell boundary (s, theta, phi, the poles):
    # the GPU's correctly rounded path must equal the oracle bit for bit, and the
    # evaluation path of each precision (FP64 estimates; FP32 angle decisions with a
    # margin) must equal both
    wl, pts, _ = _make((3000, 8, 6, 1, 2))
    g = pkg.Plan(pts, wl.kappa, 6, 3, 5, 1, 2, precision=precision)
    o = oracle.Plan(pts, wl.kappa, 6, 3, 5, 1, 2)
    rng = np.random.default_rng(5)
    for d in range(3, 7):
        lp = o.level_params(d)
        li = o.level_info(d)
        ns, nc = li["ns"], li["nc"]
        vecs = []
        eps = [0.0, 1e-16, -1e-16, 1e-14, -1e-14, 1e-12, -1e-12, 1e-11, -1e-11, 1e-9, -1e-9,
               1e-7, -1e-7, 1e-6, -1e-6, 3e-6, -3e-6, 1e-5, -1e-5]
        for _ in range(600):
            m = rng.integers(0, ns + 1)
            k = rng.integers(0, nc + 1)
            j = rng.integers(0, 2 * nc + 1)
            e = rng.choice(eps, size=3)
            s = max(m, 0.05) * lp["ds"] * (1 + e[0])
            th = k * lp["dth"] * (1 + e[1]) if k else abs(e[1])
            ph = j * lp["dth"] * (1 + e[2])
            r = lp["h"] / s
            vecs.append([r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)])
        vecs += [[0, 0, 3 * lp["H"]], [0, 0, -3 * lp["H"]], [1e-300, 0, 2 * lp["H"]]]
        vecs = np.array(vecs)
        ex, fa = g.cone_ids(d, vecs)
        ref = np.array([o.cone_of(d, v, np.zeros(3))[0][3] for v in vecs])
        assert np.array_equal(ex, ref), d
        assert np.array_equal(fa, ref), d


@pytest.mark.parametrize("nrhs", [2, 8, 64])
def test_batched_tensor_core_path_matches_mixed_and_oracle(pkg, torch_cuda, nrhs):
    # BF16 hi+lo operands keep ~16 significant bits: the contraction error is
    # ~2^-16 times the Lebesgue constant of the 3x5x5 interpolant (< 10), so 2e-4
    # relative l2 against the FP32 path; and <= 1e-3 against the direct sum
    torch = torch_cuda
    wl, pts, _ = _make((4000, 4, 5, 1, 2))
    sig = wi.complex_normal(60 + nrhs, (nrhs, wl.n))
    b = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 5, 3, 5, 1, 2, max_nrhs=nrhs, precision="batched")
    m = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 5, 3, 5, 1, 2, max_nrhs=nrhs, precision="mixed")
    s = torch.from_numpy(sig).cuda()
    ub = b.apply(s).cpu().numpy()
    um = m.apply(s).cpu().numpy()
    assert b.check() == 0
    # without the plan-time target geometry cache the result is the same
    b2 = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 5, 3, 5, 1, 2, max_nrhs=nrhs, precision="batched",
                  flags=4)
    assert rel(b2.apply(s).cpu().numpy(), ub) < 1e-5
    assert b2.check() == 0
    for r in range(nrhs):
        assert rel(ub[r], um[r]) < 2e-4, (r, rel(ub[r], um[r]))
    # stage-wise: near field only is exact FP32 work, far field alone
    assert rel(b.apply_partial(s, 1).cpu().numpy(), m.apply_partial(s, 1).cpu().numpy()) < 1e-6
    assert rel(b.apply_partial(s, 2).cpu().numpy(), m.apply_partial(s, 2).cpu().numpy()) < 2e-4
    ex = oracle.direct(pts, wl.kappa, sig[:2])
    for r in range(2):
        assert rel(ub[r], ex[r]) < 1e-3
    assert b.check() == 0


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6), ("batched", 1e-5)])
def test_two_level_buffers_and_rhs_chunks_match(pkg, torch_cuda, precision, tol):
    # flags bit 3: only two levels' cone values resident; bit 4: 2 right-hand sides
    # per pass.  Same operator, same result.
    torch = torch_cuda
    wl, pts, _ = _make((3500, 4, 5, 1, 2))
    nrhs = 6
    sig = wi.complex_normal(70, (nrhs, wl.n))
    kw = dict(max_nrhs=nrhs, precision=precision)
    a = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 5, 3, 5, 1, 2, **kw)
    b = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 5, 3, 5, 1, 2, flags=8 | 16, **kw)
    assert b.stats()["pingpong"] == 1 and b.stats()["rhs_chunk"] == 2
    assert a.stats()["pingpong"] == 0
    s = torch.from_numpy(sig).cuda()
    ua, ub = a.apply(s).cpu().numpy(), b.apply(s).cpu().numpy()
    assert rel(ub, ua) < tol
    wa, wb = a.apply_adjoint(s).cpu().numpy(), b.apply_adjoint(s).cpu().numpy()
    assert rel(wb, wa) < tol
    # a budget too small for all levels switches to two levels by itself
    eb = 16 if precision == "fp64" else 8
    lv = {x["d"]: x["nact"] * 75 * eb for x in a.stats()["level"] if x["d"] >= 3}
    pair = max(lv[d] + lv[d - 1] for d in range(4, 6))
    budget = int(1.5 * pair)
    assert sum(lv.values()) * nrhs > budget
    c = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 5, 3, 5, 1, 2, value_budget_bytes=budget, **kw)
    assert c.stats()["pingpong"] == 1
    assert rel(c.apply(s).cpu().numpy(), ua) < tol
    assert a.check() == 0 and b.check() == 0 and c.check() == 0


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_adjoint_with_just_in_time_lists(pkg, torch_cuda, precision, tol):
    # two-level plans build the adjoint's transpose lists level by level right before
    # use; flags bit 6 cuts the upward lists into ranges of at most 4096 evaluations,
    # so every level runs as many ranges; bit 4: 2 right-hand sides per pass
    torch = torch_cuda
    wl, pts, _ = _make((3500, 4, 5, 1, 2))
    nrhs = 3
    v = wi.complex_normal(71, (nrhs, wl.n))
    s = wi.complex_normal(72, (nrhs, wl.n))
    o = oracle.Plan(pts, wl.kappa, 5, 3, 5, 1, 2)
    g = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 5, 3, 5, 1, 2, max_nrhs=nrhs, precision=precision,
                 flags=8 | 16 | 64)
    assert g.stats()["pingpong"] == 1
    w = g.apply_adjoint(torch.from_numpy(v).cuda()).cpu().numpy()
    assert rel(w, o.apply_adjoint(v)) < tol
    # the adjoint identity <v, A s> = <A^H v, s> with the same plan's forward
    u = g.apply(torch.from_numpy(s).cuda()).cpu().numpy()
    lhs, rhs = np.vdot(v, u), np.vdot(w, s)
    assert abs(lhs - rhs) / abs(lhs) < (1e-12 if precision == "fp64" else 1e-5)
    # profiled: the list building and the adjoint launches of every range are timed, and
    # the result does not change
    g.set_profiling(True)
    w2 = g.apply_adjoint(torch.from_numpy(v).cuda()).cpu().numpy()
    tm = g.timings()
    g.set_profiling(False)
    assert np.array_equal(w2, w)
    st = tm["stages"]
    assert tm["calls"] == 1
    assert st["adj_level"]["launches"] > 4 and st["adj_level"]["ms"] > 0  # many ranges (bit 6)
    assert st["adj_lists"]["ms"] > 0 and st["adj_eval"]["launches"] >= 2  # two chunks' near fields
    assert st["permute_in"]["launches"] == 2 and st["permute_out"]["launches"] == 2
    assert g.check() == 0


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("mixed", 1e-6)])
def test_evaluation_caches_match_on_the_fly_geometry(pkg, torch_cuda, precision, tol):
    # plan-time caches of cousin-target and untabled-upward geometry (default) vs none
    # (flags bit 5), and vs the oracle; both ping-pong and resident levels
    torch = torch_cuda
    wl, pts, sigma = _make((5000, 4, 6, 1, 2))
    s = torch.from_numpy(sigma).cuda()
    o = oracle.Plan(pts, wl.kappa, 6, 3, 5, 1, 2)
    uo = o.apply(sigma)
    for extra in (0, 8):
        a = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 6, 3, 5, 1, 2, precision=precision, flags=extra)
        b = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 6, 3, 5, 1, 2, precision=precision, flags=32 | extra)
        assert a.stats()["cache_bytes"] > 0 and b.stats()["cache_bytes"] == 0
        ua, ub = a.apply(s).cpu().numpy(), b.apply(s).cpu().numpy()
        assert rel(ua, ub) < tol
        assert rel(ua, uo) < (1e-10 if precision == "fp64" else 2e-5)
        # the adjoint reads the same caches (resident plans: the target cache through
        # the transpose lists' cache indices; both: the untabled upward cache)
        wa, wb = a.apply_adjoint(s).cpu().numpy(), b.apply_adjoint(s).cpu().numpy()
        assert rel(wa, wb) < tol
        assert rel(wa, o.apply_adjoint(sigma)) < (1e-10 if precision == "fp64" else 2e-5)
        assert a.check() == 0 and b.check() == 0


def test_host_pointer_path_matches_device_path(pkg, torch_cuda):
    torch = torch_cuda
    wl, pts, sigma = _make((2000, 2, 4, 1, 2))
    g = pkg.Plan(pts, wl.kappa, 4, 3, 5, 1, 2)
    u_host = g.apply(sigma)
    u_dev = g.apply(torch.from_numpy(sigma).cuda()).cpu().numpy()
    assert np.array_equal(u_host, u_dev)
    # bitwise reproducible run to run
    assert np.array_equal(g.apply(sigma), u_host)
    w1 = g.apply_adjoint(sigma)
    assert np.array_equal(g.apply_adjoint(sigma), w1)


LEAF = ["16x8", "32x4", "8x16"]


@pytest.mark.parametrize("nrhs", [2, 24, 64])
def test_autotuned_tile_shapes_give_the_same_result(pkg, torch_cuda, nrhs):
    # every leaf tile shape sums each output over the sources in the same order, and the
    # cone grid only changes which CTA takes which cone: same leaf values, same field
    # up to the run-to-run order of the cone kernel's FP32 reductions
    torch = torch_cuda
    wl, pts, _ = _make((4000, 4, 5, 1, 2))
    sig = wi.complex_normal(110 + nrhs, (nrhs, wl.n))
    b = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 5, 3, 5, 1, 2, max_nrhs=nrhs, precision="batched")
    s = torch.from_numpy(sig).cuda().to(torch.complex64)
    u0 = b.apply(s).cpu().numpy()
    leaf0 = b.values(5, nrhs)
    for shape in range(3):
        for ctas in (1, 2):
            b.set_tiles(shape, ctas)
            u = b.apply(s).cpu().numpy()
            assert rel(u, u0) < 1e-5, (shape, ctas, rel(u, u0))
            lv = b.values(5, nrhs)
            assert rel(lv, leaf0) < 1e-6, (shape, rel(lv, leaf0))
    tune = b.autotune(nrhs, reps=2)
    assert tune["leaf_shape"] in ("16x8", "32x4", "8x16") and tune["cone_ctas_per_sm"] in (1, 2)
    assert all(t > 0 for t in tune["leaf_ms"] + tune["cone_ms"])
    st = b.stats()
    assert ["16x8", "32x4", "8x16"][st["tune_leaf"]] == tune["leaf_shape"]
    assert st["tune_cone_ctas"] == tune["cone_ctas_per_sm"]
    # the tuner's runs use the plan's own buffers: the caller's field is unchanged
    assert rel(b.apply(s).cpu().numpy(), u0) < 1e-5
    ex = oracle.direct(pts, wl.kappa, sig[:1])
    assert rel(b.apply(s).cpu().numpy()[:1], ex) < 1e-3
    with pytest.raises(pkg.IFGFError):
        b.autotune(3)
    with pytest.raises(pkg.IFGFError):
        b.set_tiles(3, 1)
    assert b.check() == 0


def test_tune_cache_reuses_a_choice_across_plans(pkg, torch_cuda, tmp_path):
    # the first plan of a workload is timed and its choice appended to the cache file; a
    # second plan of the same workload takes the choice from the file without timing; a
    # plan of another nrhs is a different key
    torch = torch_cuda
    wl, pts, _ = _make((4000, 4, 5, 1, 2))
    path = str(tmp_path / "tune.txt")
    x = torch.from_numpy(pts).cuda()
    b1 = pkg.Plan(x, wl.kappa, 5, 3, 5, 1, 2, max_nrhs=16, precision="batched")
    t1 = b1.autotune(16, reps=1, cache=path)
    assert not t1["cached"] and " " not in t1["key"]
    assert open(path).read().split() == [t1["key"], str(LEAF.index(t1["leaf_shape"])), str(t1["cone_ctas_per_sm"])]
    b2 = pkg.Plan(x, wl.kappa, 5, 3, 5, 1, 2, max_nrhs=16, precision="batched")
    assert b2.tune_key(16) == t1["key"]
    b2.set_tiles((LEAF.index(t1["leaf_shape"]) + 1) % 3, 3 - t1["cone_ctas_per_sm"])  # not the cached shapes
    t2 = b2.autotune(16, reps=1, cache=path)
    assert t2["cached"] and t2["leaf_shape"] == t1["leaf_shape"] and t2["cone_ctas_per_sm"] == t1["cone_ctas_per_sm"]
    st = b2.stats()
    assert LEAF[st["tune_leaf"]] == t1["leaf_shape"] and st["tune_cone_ctas"] == t1["cone_ctas_per_sm"]
    assert b2.tune_key(8) != t1["key"]
    t3 = b2.autotune(8, reps=1, cache=path)
    assert not t3["cached"] and len(open(path).read().splitlines()) == 2
    with pytest.raises(pkg.IFGFError):
        b2.autotune(3, cache=path)  # odd nrhs: rejected even though nothing is cached for it
    s = torch.from_numpy(wi.complex_normal(7, (16, wl.n))).cuda().to(torch.complex64)
    assert rel(b2.apply(s).cpu().numpy(), b1.apply(s).cpu().numpy()) < 1e-5
    assert b1.check() == 0 and b2.check() == 0


@pytest.mark.parametrize("precision,nrhs,flags", [("fp64", 1, 0), ("mixed", 3, 0), ("batched", 4, 0),
                                                   ("fp64", 2, 8 | 16)])
def test_graph_replay_matches_plain_launches(pkg, torch_cuda, precision, nrhs, flags):
    # a captured evaluation replays the same kernels in the same order: bitwise equal
    # results on the deterministic paths, and new buffer contents are picked up
    torch = torch_cuda
    wl, pts, _ = _make((3000, 4, 5, 1, 2))
    sig = wi.complex_normal(90 + nrhs, (2, nrhs, wl.n))
    g = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 5, 3, 5, 1, 2, max_nrhs=nrhs, precision=precision,
                 flags=flags)
    s = torch.from_numpy(sig[0]).cuda().to(g.complex_dtype)
    plain = [g.apply(s).cpu().numpy(), g.apply_adjoint(s).cpu().numpy()]
    s2 = torch.from_numpy(sig[1]).cuda().to(g.complex_dtype)
    plain2 = g.apply(s2).cpu().numpy()
    g.set_graphs(True)
    u = torch.empty_like(s)
    w = torch.empty_like(s)
    got = []
    for _ in range(3):
        g.apply(s, out=u)
        g.apply_adjoint(s, out=w)
        got.append((u.cpu().numpy(), w.cpu().numpy()))
    s.copy_(s2)
    g.apply(s, out=u)
    got2 = u.cpu().numpy()
    # host buffers go through the plan's staging buffers: one more graph
    uh = g.apply(sig[1].astype(g.numpy_dtype))
    st = g.stats()
    pingpong_adjoint = bool(flags & 8)   # adjoint lists built between launches: not captured
    assert st["graph_captures"] == (2 if pingpong_adjoint else 3)
    assert st["graph_replays"] == (5 if pingpong_adjoint else 8)
    exact = precision != "batched"
    for uu, ww in got:
        if exact:
            assert np.array_equal(uu, plain[0])
            assert np.array_equal(ww, plain[1])
        else:
            assert rel(uu, plain[0]) < 1e-5
            assert rel(ww, plain[1]) < 1e-5
    if exact:
        assert np.array_equal(got2, plain2)
        assert np.array_equal(uh, plain2)
    else:
        assert rel(got2, plain2) < 1e-5
        assert rel(uh, plain2) < 1e-5
    # with profiling on, the graph records the stage events: stage times add up to
    # the call and the result does not change
    g.set_profiling(True)
    for _ in range(2):
        g.apply(s, out=u)
    tm = g.timings()
    g.set_profiling(False)
    assert tm["calls"] == 2
    assert sum(v["ms"] for v in tm["stages"].values()) > 0
    assert tm["stages"]["upward"]["launches"] > 0
    if exact:
        assert np.array_equal(u.cpu().numpy(), plain2)
    assert g.stats()["graph_captures"] == (3 if pingpong_adjoint else 4)
    g.set_graphs(False)
    assert g.stats()["graphs"] == 0
    assert g.check() == 0


@pytest.mark.parametrize("case", CASES[:3])
def test_mixed_precision_matches_fp64_oracle(pkg, torch_cuda, case):
    torch = torch_cuda
    wl, pts, sigma = _make(case)
    n, nl, D, ns, nc = case
    g = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, D, 3, 5, ns, nc, precision="mixed")
    o = oracle.Plan(pts, wl.kappa, D, 3, 5, ns, nc)
    u = g.apply(torch.from_numpy(sigma).cuda()).cpu().numpy()
    assert rel(u, o.apply(sigma)) < 2e-5
    v = wi.complex_normal(7, (1, n))
    w = g.apply_adjoint(torch.from_numpy(v).cuda()).cpu().numpy()
    assert rel(w, o.apply_adjoint(v)) < 2e-5
    assert g.check() == 0


def test_mixed_near_field_close_pairs(pkg, torch_cuda):
    # Float plans form near-field distances in FP32 from split leaf offsets; the
    # difference of the high parts is exact for close pairs, so pairs 1e-7 of a leaf
    # box apart keep FP32 relative accuracy (a plain FP32 difference of the offsets
    # would be off by tens of percent there).
    torch = torch_cuda
    wl, pts, _ = _make((3000, 3, 4, 2, 4))
    H = (pts.max(0) - pts.min(0)).max() / 2 ** 3
    rng = np.random.default_rng(5)
    dirs = rng.normal(size=(3, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    extra = pts[[10, 500, 2000]] + 1e-7 * H * dirs
    allp = np.ascontiguousarray(np.vstack([pts, extra]))
    n = allp.shape[0]
    sigma = wi.complex_normal(21, (1, n))
    g = pkg.Plan(torch.from_numpy(allp).cuda(), wl.kappa, 4, 3, 5, 2, 4, precision="mixed")
    o = oracle.Plan(allp, wl.kappa, 4, 3, 5, 2, 4)
    un = g.apply_partial(torch.from_numpy(sigma.astype(np.complex64)).cuda(), 1).cpu().numpy()
    ref = o.apply(sigma, mode=1)
    assert rel(un, ref) < 2e-5
    close = [10, 500, 2000, n - 3, n - 2, n - 1]
    err = np.abs(un[0, close] - ref[0, close]) / np.abs(ref[0, close])
    assert err.max() < 1e-5, err
    w = g.apply_adjoint(torch.from_numpy(sigma.astype(np.complex64)).cuda()).cpu().numpy()
    assert rel(w, o.apply_adjoint(sigma)) < 2e-5
    assert g.check() == 0


def test_duplicate_points_rejected(pkg, torch_cuda):
    # the points must be pairwise distinct: an exact duplicate is an invalid argument,
    # a point 1e-13 away from another is accepted
    torch = torch_cuda
    wl, pts, _ = _make((3000, 3, 4, 2, 4))
    dup = np.ascontiguousarray(np.vstack([pts, pts[17:18]]))
    with pytest.raises(pkg.IFGFError) as ei:
        pkg.Plan(torch.from_numpy(dup).cuda(), wl.kappa, 4, 3, 5, 2, 4)
    assert "duplicate" in str(ei.value)
    near = dup.copy()
    near[-1, 0] += 1e-13
    g = pkg.Plan(torch.from_numpy(near).cuda(), wl.kappa, 4, 3, 5, 2, 4)
    assert g.stats()["n"] == near.shape[0]


def test_host_wait_timeout_is_reported(pkg, torch_cuda):
    # flags bit 7: the host-side wait never sees the device finish (a fake of the event
    # query), so an evaluation with host buffers returns IFGF_ETIMEOUT after timeout_s;
    # the queued work completes on its own and the device stays usable
    torch = torch_cuda
    wl, pts, sigma = _make((3000, 3, 4, 2, 4))
    dpts = torch.from_numpy(pts).cuda()
    g = pkg.Plan(dpts, wl.kappa, 4, 3, 5, 2, 4, flags=128, timeout_s=0.05)
    with pytest.raises(pkg.IFGFError) as ei:
        g.apply(sigma)  # numpy in and out: the call waits for its result
    assert ei.value.status == 4
    torch.cuda.synchronize()
    h = pkg.Plan(dpts, wl.kappa, 4, 3, 5, 2, 4, timeout_s=30.0)
    u = h.apply(sigma)  # a bounded wait that succeeds
    u = u if isinstance(u, np.ndarray) else u.cpu().numpy()
    ref = h.apply(torch.from_numpy(sigma).cuda()).cpu().numpy()
    assert np.array_equal(u, ref)
    assert g.check() == 0 and h.check() == 0


def test_device_wait_limit_reports_error(pkg, torch_cuda):
    # flags bit 8: the tensor-core cone kernel issues no MMA, so each CTA's bounded wait
    # for its MMAs runs out (shortened limit); the kernel counts it in the device error
    # counter, frees its tensor memory and returns, and the device stays usable
    torch = torch_cuda
    wl, pts, _ = _make((4000, 4, 5, 1, 2))
    nrhs = 4
    s = torch.from_numpy(wi.complex_normal(73, (nrhs, wl.n))).cuda()
    dpts = torch.from_numpy(pts).cuda()
    bad = pkg.Plan(dpts, wl.kappa, 5, 3, 5, 1, 2, max_nrhs=nrhs, precision="batched", flags=256)
    bad.apply(s)
    assert bad.check() > 0
    good = pkg.Plan(dpts, wl.kappa, 5, 3, 5, 1, 2, max_nrhs=nrhs, precision="batched")
    m = pkg.Plan(dpts, wl.kappa, 5, 3, 5, 1, 2, max_nrhs=nrhs, precision="mixed")
    assert rel(good.apply(s).cpu().numpy(), m.apply(s).cpu().numpy()) < 2e-4
    assert good.check() == 0 and m.check() == 0


def test_autograd_gradient_matches_finite_differences(pkg, torch_cuda):
    # L = ||A sigma||^2 is quadratic, so central differences are exact up to rounding
    torch = torch_cuda
    wl, pts, sigma = _make((3000, 4, 4, 2, 4))
    g = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 4, 3, 5, 2, 4)
    s = torch.from_numpy(sigma[0]).cuda().requires_grad_(True)
    u = pkg.ifgf_apply_autograd(s[None, :], g)
    loss = (u.abs() ** 2).sum()
    loss.backward()
    grad = s.grad.cpu().numpy()
    idx = wi.sample_targets(wl.n, 16, 300)
    h = 1e-3
    base = sigma[0].copy()

    def L(x):
        return float((np.abs(g.apply(torch.from_numpy(x[None, :]).cuda()).cpu().numpy()) ** 2).sum())

    for m in idx:
        for part, unit in ((0, 1.0), (1, 1j)):
            xp = base.copy(); xp[m] += h * unit
            xm = base.copy(); xm[m] -= h * unit
            fd = (L(xp) - L(xm)) / (2 * h)
            an = grad[m].real if part == 0 else grad[m].imag
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)) + 1e-6 * np.abs(grad).max(), (m, part, fd, an)


# ------------------------------------------------------------------------------------
# Element-wise bounds.  ELEM_* bound max_i |a_i - b_i| / max_i |b_i| for one right-hand
# side: every output, scaled by the field's largest value (a relative bound per element
# is not defined where the field passes near zero).
#   * mixed (FP32 values, FP64 geometry): each output sums ~10^3 FP32-rounded terms per
#     level (unit roundoff 6e-8) whose magnitudes reach a few times max|u|, through
#     interpolants of Lebesgue constant below 8: 1e-4.
#   * batched (BF16 hi+lo operands, FP32 accumulate): each operand keeps 16 significant
#     bits (relative error 2^-17 per operand, 2^-16 for the dropped lo*lo term), which
#     the interpolant's Lebesgue constant (< 8) and the up to 7 levels carry to the
#     outputs: 2e-3 per element, and 2e-4 relative l2 per right-hand side.
# ------------------------------------------------------------------------------------
ELEM_MIXED = 1e-4
ELEM_BATCHED = 2e-3


def _tree_and_cones_equal(g, o, D):
    H1, corner = g.geometry()
    oH1, ocorner = o.geometry()
    assert H1 == oH1 and np.array_equal(corner, ocorner)
    assert np.array_equal(g.perm(), o.perm())
    for d in range(1, D + 1):
        gk, gs = g.boxes(d)
        ok, os_ = o.boxes(d)
        assert np.array_equal(gk, ok) and np.array_equal(gs, os_), d
    for d in range(3, D + 1):
        gs, gl = g.cousins(d)
        os_, ol = o.cousins(d)
        assert np.array_equal(gs, os_) and np.array_equal(gl, ol), d
        ga, gc = g.active(d)
        oa, oc = o.active(d)
        assert np.array_equal(ga, oa) and np.array_equal(gc, oc), d


@pytest.mark.parametrize("kind", wi.DEGENERATE)
def test_degenerate_geometries_match_oracle(pkg, torch_cuda, kind):
    # two points, collinear points, a flat disc and two far-apart clusters: bounding
    # cubes with zero extent along some axes, clamped integer coordinates, points on the
    # cone axes and mostly empty boxes.  Tree and cones bit-exact; FP64 forward and
    # adjoint to 1e-10 of the oracle's IFGF, mixed to the element-wise FP32 bound.
    torch = torch_cuda
    pts, kappa, D = wi.degenerate_points(kind)
    n = len(pts)
    dp = torch.from_numpy(pts).cuda()
    g = pkg.Plan(dp, kappa, D, 3, 5, 1, 2)
    o = oracle.Plan(pts, kappa, D, 3, 5, 1, 2)
    _tree_and_cones_equal(g, o, D)
    sig = wi.complex_normal(5, (1, n))
    v = wi.complex_normal(6, (1, n))
    uo, wo = o.apply(sig), o.apply_adjoint(v)
    u = g.apply(torch.from_numpy(sig).cuda()).cpu().numpy()
    w = g.apply_adjoint(torch.from_numpy(v).cuda()).cpu().numpy()
    assert maxrel(u, uo) < 1e-10, maxrel(u, uo)
    assert maxrel(w, wo) < 1e-10, maxrel(w, wo)
    m = pkg.Plan(dp, kappa, D, 3, 5, 1, 2, precision="mixed")
    um = m.apply(torch.from_numpy(sig).cuda()).cpu().numpy()
    wm = m.apply_adjoint(torch.from_numpy(v).cuda()).cpu().numpy()
    assert maxrel(um, uo) < ELEM_MIXED, maxrel(um, uo)
    assert maxrel(wm, wo) < ELEM_MIXED, maxrel(wm, wo)
    assert g.check() == 0 and m.check() == 0


@pytest.mark.parametrize("case", CASES[:3])
def test_mixed_elementwise_vs_oracle(pkg, torch_cuda, case):
    # the mixed path, forward and adjoint, every output against the FP64 oracle IFGF
    torch = torch_cuda
    wl, pts, _ = _make(case)
    n, nl, D, ns, nc = case
    sig = wi.complex_normal(80, (3, n))
    g = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, D, 3, 5, ns, nc, precision="mixed", max_nrhs=3)
    o = oracle.Plan(pts, wl.kappa, D, 3, 5, ns, nc)
    s = torch.from_numpy(sig).cuda()
    u, uo = g.apply(s).cpu().numpy(), o.apply(sig)
    w, wo = g.apply_adjoint(s).cpu().numpy(), o.apply_adjoint(sig)
    for r in range(3):
        assert maxrel(u[r], uo[r]) < ELEM_MIXED, (r, maxrel(u[r], uo[r]))
        assert maxrel(w[r], wo[r]) < ELEM_MIXED, (r, maxrel(w[r], wo[r]))
    assert g.check() == 0


@pytest.mark.parametrize("precision,elem,l2", [("batched", ELEM_BATCHED, 2e-4), ("batched_fp16", ELEM_MIXED, 2e-5)])
@pytest.mark.parametrize("nrhs", [2, 16, 64])
def test_batched_every_rhs_elementwise_vs_oracle(pkg, torch_cuda, nrhs, precision, elem, l2):
    # the tensor-core path against the FP64 oracle IFGF, right-hand side by right-hand
    # side: every output within the element-wise bound and each field within the l2
    # bound of its operand type (BF16 hi + lo keeps ~16 bits: ELEM_BATCHED, 2e-4; FP16
    # hi + lo with per-cone scaling keeps ~22 bits, as fine as FP32 accumulation over the
    # levels allows: ELEM_MIXED, 2e-5); the adjoint (run by the mixed kernels) within
    # ELEM_MIXED
    torch = torch_cuda
    wl, pts, _ = _make((4000, 4, 5, 1, 2))
    sig = wi.complex_normal(160 + nrhs, (nrhs, wl.n))
    b = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 5, 3, 5, 1, 2, max_nrhs=nrhs, precision=precision)
    o = oracle.Plan(pts, wl.kappa, 5, 3, 5, 1, 2)
    s = torch.from_numpy(sig).cuda()
    ub, uo = b.apply(s).cpu().numpy(), o.apply(sig)
    for r in range(nrhs):
        assert maxrel(ub[r], uo[r]) < elem, (r, maxrel(ub[r], uo[r]))
        assert rel(ub[r], uo[r]) < l2, (r, rel(ub[r], uo[r]))
    wb, wo = b.apply_adjoint(s).cpu().numpy(), o.apply_adjoint(sig)
    for r in range(nrhs):
        assert maxrel(wb[r], wo[r]) < ELEM_MIXED, (r, maxrel(wb[r], wo[r]))
    assert b.check() == 0


@pytest.mark.parametrize("nrhs,flags", [(1, 0), (2, 0), (3, 0), (4, 0), (4, 2), (4, 8 | 32), (4, 1024),
                                        (1, 2 | 1024), (4, 2 | 2048), (3, 8 | 32 | 2048), (6, 0), (8, 0),
                                        (7, 2 | 1024)])
def test_run_fp32_upward_matches_l1_kernel(pkg, torch_cuda, nrhs, flags):
    # the FP32 upward step in runs of nodes that share a child cone (default) and the
    # kernel with one thread per parent node reading the values from L1 (flags bit 9) sum
    # every parent node over the same children in the same order; the run kernel
    # associates each 75-term contraction differently (weight products), so the cone
    # values agree to FP32 rounding carried over the levels (1e-5, a tenth of the mixed
    # path's element-wise bound); tabled (default) and on-the-fly geometry (bit 1);
    # two-level buffers without caches (bits 3 and 5); runs taken by 8 lanes (bit 10);
    # more than 4 right-hand sides: the run kernel on blocks of 4 (6 = 4 + 2, 7 = 4 + 3)
    torch = torch_cuda
    wl, pts, _ = _make((6000, 6, 6, 1, 2))
    sig = wi.complex_normal(200 + nrhs, (nrhs, wl.n))
    kw = dict(max_nrhs=nrhs, precision="mixed")
    a = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 6, 3, 5, 1, 2, flags=flags, **kw)
    b = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 6, 3, 5, 1, 2, flags=flags | 512, **kw)
    s = torch.from_numpy(sig).cuda().to(torch.complex64)
    ua, ub = a.apply(s).cpu().numpy(), b.apply(s).cpu().numpy()
    assert maxrel(ua, ub) < 1e-5, maxrel(ua, ub)
    if not flags & 8:
        for d in range(3, 7):
            va, vb = a.values(d, nrhs), b.values(d, nrhs)
            assert maxrel(va, vb) < 1e-5, (d, maxrel(va, vb))
    o = oracle.Plan(pts, wl.kappa, 6, 3, 5, 1, 2)
    uo = o.apply(sig)
    for r in range(nrhs):
        assert maxrel(ua[r], uo[r]) < ELEM_MIXED, (r, maxrel(ua[r], uo[r]))
    assert a.check() == 0 and b.check() == 0


@pytest.mark.parametrize("nrhs,flags", [(1, 0), (1, 2), (1, 1024), (1, 2 | 2048), (2, 0), (4, 0), (6, 1024)])
def test_run_fp32_upward_order_4_7_matches_l1_kernel(pkg, torch_cuda, nrhs, flags):
    # (P_s, P_ang) = (4, 7): a child step of 196 nodes has more than 32 runs, so lanes take
    # several runs each; 2 and 4 right-hand sides take 53 KB of shared memory per CTA (above
    # the default limit); 6 run as blocks of 4 + 2; same comparison as at (3, 5)
    torch = torch_cuda
    wl, pts, _ = _make((4000, 4, 5, 1, 2))
    sig = wi.complex_normal(210 + nrhs, (nrhs, wl.n))
    kw = dict(max_nrhs=nrhs, precision="mixed")
    a = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 5, 4, 7, 1, 2, flags=flags, **kw)
    b = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 5, 4, 7, 1, 2, flags=flags | 512, **kw)
    s = torch.from_numpy(sig).cuda().to(torch.complex64)
    ua, ub = a.apply(s).cpu().numpy(), b.apply(s).cpu().numpy()
    assert maxrel(ua, ub) < 1e-5, maxrel(ua, ub)
    for d in range(3, 6):
        va, vb = a.values(d, nrhs), b.values(d, nrhs)
        assert maxrel(va, vb) < 1e-5, (d, maxrel(va, vb))
    uo = oracle.Plan(pts, wl.kappa, 5, 4, 7, 1, 2).apply(sig)
    for r in range(nrhs):
        assert maxrel(ua[r], uo[r]) < ELEM_MIXED, (r, maxrel(ua[r], uo[r]))
    assert a.check() == 0 and b.check() == 0


@pytest.mark.parametrize("precision,elem,l2", [("batched", ELEM_BATCHED, 2e-4), ("batched_fp16", ELEM_MIXED, 2e-5)])
@pytest.mark.parametrize("nrhs", [2, 16, 48])
def test_batched_order_4_7_vs_oracle(pkg, torch_cuda, nrhs, precision, elem, l2):
    # (P_s, P_ang) = (4, 7) on the tensor cores: 196 nodes per cone, contraction length 208
    # (13 K blocks), one CTA per SM at 48 right-hand sides; every right-hand side against
    # the oracle's order-(4, 7) IFGF element-wise, and the first against the direct sum
    torch = torch_cuda
    wl, pts, _ = _make((3000, 3, 4, 2, 4))
    sig = wi.complex_normal(300 + nrhs, (nrhs, wl.n))
    b = pkg.Plan(torch.from_numpy(pts).cuda(), wl.kappa, 4, 4, 7, 2, 4, max_nrhs=nrhs, precision=precision)
    o = oracle.Plan(pts, wl.kappa, 4, 4, 7, 2, 4)
    s = torch.from_numpy(sig).cuda()
    ub, uo = b.apply(s).cpu().numpy(), o.apply(sig)
    for r in range(nrhs):
        assert maxrel(ub[r], uo[r]) < elem, (r, maxrel(ub[r], uo[r]))
        assert rel(ub[r], uo[r]) < l2, (r, rel(ub[r], uo[r]))
    ex = oracle.direct(pts, wl.kappa, sig[:1])
    assert rel(ub[:1], ex) < 1e-3
    tune = b.autotune(nrhs, reps=1)
    assert tune["cone_ctas_per_sm"] in (1, 2)
    assert rel(b.apply(s).cpu().numpy(), ub) < 1e-5
    assert b.check() == 0
