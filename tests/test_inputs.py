"""Pins for the seeded input generators (ifgf_inputs), which feed both the oracle and the
CUDA path: the random streams against published values and their moments, and every
surface sampler against its surface equation and, for the area-uniform ones, against
areas computed independently (quadrature, face areas).
"""
import math

import numpy as np
import pytest

import ifgf_inputs as wi


def test_splitmix64_matches_published_outputs():
    # SplitMix64 with state 0 (Steele, Lea & Flood 2014; Java's SplittableRandom(0)
    # gives -2152535657050944081 as its first nextLong): the first three outputs
    out = [int(v) for v in wi.splitmix64(0, 0, 3)]
    assert out[0] == 0xE220A8397B1DCDAF == (1 << 64) - 2152535657050944081
    assert out[1:] == [0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # counter-based: any window of a stream is the same slice of the whole stream
    assert np.array_equal(wi.splitmix64(9, 5, 4), wi.splitmix64(9, 0, 9)[5:])


def test_uniform_and_normal_moments():
    n = 200_000
    u = wi.uniform(123, 0, n)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 0.002
    z = wi.normal(321, n)
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 0.015
    assert abs(np.mean(z ** 4) - 3.0) < 0.06          # Gaussian kurtosis
    c = wi.complex_normal(7, (3, 50_000))
    assert c.dtype == np.complex128 and c.shape == (3, 50_000)
    assert abs(np.mean(c.real ** 2) - 1) < 0.03 and abs(np.mean(c.imag ** 2) - 1) < 0.03
    assert abs(np.mean(c.real * c.imag)) < 0.02       # independent parts


def test_fibonacci_sphere_closed_form():
    n = 4096
    p = wi.fibonacci_sphere(n)
    assert np.max(np.abs(np.linalg.norm(p, axis=1) - 1.0)) < 1e-15
    i = np.arange(n)
    assert np.array_equal(p[:, 2], 1.0 - (2.0 * i + 1.0) / n)
    assert np.max(np.abs(p.mean(axis=0))) < 1e-3      # no point exactly at a pole, balanced
    assert len(np.unique(p, axis=0)) == n


def test_prolate_spheroid_points_are_area_uniform():
    a, c = 0.1, 1.0
    n = 100_000
    p = wi.spheroid_points(n, axes=(a, a, c), seed=3)
    assert p.shape == (n, 3)
    assert np.max(np.abs(p[:, 0] ** 2 / a ** 2 + p[:, 1] ** 2 / a ** 2 + p[:, 2] ** 2 / c ** 2 - 1.0)) < 1e-12
    # surface of revolution: dA / dz = 2 pi sqrt(rho^2 + (rho rho')^2), rho^2 = a^2 (1 - z^2 / c^2)
    zs = np.linspace(-c, c, 200_001)
    dens = np.sqrt(a * a * (1 - zs ** 2 / c ** 2) + (a * a * zs / c ** 2) ** 2)
    for z0 in (0.25, 0.5, 0.9):
        band = np.abs(zs) < z0
        frac = np.trapezoid(dens * band, zs) / np.trapezoid(dens, zs)
        got = np.mean(np.abs(p[:, 2]) < z0)
        assert abs(got - frac) < 5 * math.sqrt(frac * (1 - frac) / n), (z0, got, frac)
    # azimuthally uniform
    phi = np.arctan2(p[:, 1], p[:, 0])
    assert abs(np.mean(phi > 0) - 0.5) < 5 * math.sqrt(0.25 / n)


def test_cube_union_points_lie_on_the_boundary_and_are_area_uniform():
    n = 100_000
    p = wi.cube_union_points(n)
    lo = np.array([c[0] for c in wi.CUBES])
    side = np.array([c[1] for c in wi.CUBES])
    # on a face of some cube, strictly inside none
    on_face = np.zeros(n, dtype=bool)
    for j in range(len(wi.CUBES)):
        inside = np.all((p > lo[j]) & (p < lo[j] + side[j]), axis=1)
        assert not inside.any()
        within = np.all((p >= lo[j]) & (p <= lo[j] + side[j]), axis=1)
        face = np.any((p == lo[j]) | (p == lo[j] + side[j]), axis=1)
        on_face |= within & face
    assert on_face.all()
    # the union's boundary: 3 x 2400 minus the 4 x 300 hidden by the two overlaps = 6000;
    # two fully exposed faces of area 400 each hold 400 / 6000 of the points
    for mask in (p[:, 0] == 0.0, p[:, 0] == 40.0):
        frac = 400.0 / 6000.0
        assert abs(np.mean(mask) - frac) < 5 * math.sqrt(frac * (1 - frac) / n)
    # partly hidden faces on the plane x = 20: cube 0's face loses (y, z) in [10, 20]^2 and
    # cube 2's face loses [20, 30]^2 to cube 1, leaving 300 + 300 of their 2 x 400
    frac = 600.0 / 6000.0
    assert abs(np.mean(p[:, 0] == 20.0) - frac) < 5 * math.sqrt(frac * (1 - frac) / n)


def test_sample_targets_is_a_seeded_permutation_prefix():
    n = 1000
    full = wi.sample_targets(n, n, 5)
    assert np.array_equal(np.sort(full), np.arange(n))
    assert np.array_equal(wi.sample_targets(n, 37, 5), full[:37])
    assert not np.array_equal(wi.sample_targets(n, 37, 6), full[:37])
    big = wi.sample_targets(10 ** 9, 64, 1)
    assert len(set(big.tolist())) == 64 and big.min() >= 0 and big.max() < 10 ** 9


def test_plane_wave_densities():
    pts = wi.fibonacci_sphere(500) * 3.0
    kappa, nrhs = 2.0, 5
    s = wi.plane_wave_densities(pts, kappa, nrhs, seed=4)
    assert s.shape == (nrhs, 500)
    # constant modulus per right-hand side, |A_r|
    assert np.max(np.abs(np.abs(s) - np.abs(s[:, :1]))) < 1e-12
    # a plane wave: sigma(x) conj(sigma(y)) = exp(i kappa d . (x - y)) |A|^2 with |d| = 1,
    # so the phase difference over a segment never exceeds kappa |x - y|
    ph = np.angle(s[:, 1:] * np.conj(s[:, :-1]))
    dist = np.linalg.norm(pts[1:] - pts[:-1], axis=1)
    assert np.all(np.abs(ph) <= kappa * dist[None, :] + 1e-9)


@pytest.mark.parametrize("name", sorted(wi.WORKLOADS))
def test_named_workloads_are_deterministic(name):
    wl = wi.WORKLOADS[name]
    if wl.n > 2_000_000:
        pytest.skip("large point set; determinism is covered by the smaller workloads")
    a, b = wl.points(), wl.points()
    assert a.shape == (wl.n, 3) and np.array_equal(a, b)
    assert np.all(np.isfinite(a))


def test_row_blocks_of_a_batch_are_the_batch_rows():
    # the densities a rank generates for its right-hand sides are exactly those rows of
    # the whole batch, and the first nrhs rows of a larger batch are the workload's own
    full = wi.complex_normal(41, (6, 1000))
    assert np.array_equal(wi.complex_normal_rows(41, 6, 1000, 0, 6), full)
    assert np.array_equal(wi.complex_normal_rows(41, 6, 1000, 2, 5), full[2:5])
    wl = wi.small_sphere(500, 2, 3, nrhs=2)
    assert np.array_equal(wl.densities((0, 2, 8)), wl.densities())
    assert np.array_equal(wl.densities((3, 5, 8)), wi.complex_normal(wl.seed + 100, (8, 500))[3:5])
    cubes = wi.Workload("c", 400, 1.0, 3, nrhs=4, surface="cubes", seed=4)
    assert np.allclose(cubes.densities((1, 3, 4)), cubes.densities()[1:3], rtol=0, atol=0)
