"""Seeded synthetic inputs for the IFGF operator: point sets, densities, targets.

This module is shared by the CPU oracle's tests and by the CUDA path's tests and
benchmark.  It holds only random-number and surface-sampling code, none of the
method's arithmetic (no Green function, no tree, no interpolation).

Random numbers come from the counter-based SplitMix64 generator (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
output i of stream `seed` is mix64(seed + (i + 1) * 0x9E3779B97F4A7C15), with the
published mix64 finaliser.  Uniform doubles take the top 53 bits; normal variates
use the Box-Muller transform.

Workloads (surfaces in the units of the paper's Section 4 examples):
  * Fibonacci lattice on the unit sphere (the paper's sphere of radius a = 1),
  * area-uniform points on the prolate spheroid of Eq. (defspheroid) with
    alpha = beta = 0.1, gamma = 1,
  * area-uniform points on the surface of a union of three overlapping cubes
    (not in the paper; a closed non-convex surface with sharp edges).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int) -> np.ndarray:
    """count standard normal variates (Box-Muller on consecutive uniform pairs)."""
    npair = (count + 1) // 2
    u = uniform(seed, 0, 2 * npair)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * npair)
    out[0::2] = rad * np.cos(2.0 * np.pi * u2)
    out[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return out[:count]


def complex_normal(seed: int, shape) -> np.ndarray:
    """complex128 array whose real and imaginary parts are i.i.d. N(0,1)."""
    n = int(np.prod(shape))
    z = normal(seed, 2 * n)
    return (z[0::2] + 1j * z[1::2]).reshape(shape)


def complex_normal_rows(seed: int, nrows: int, ncols: int, r0: int, r1: int) -> np.ndarray:
    """Rows r0..r1-1 of complex_normal(seed, (nrows, ncols)), generated alone.

    Element f (row-major) of that array is the Box-Muller pair of uniforms 2f and 2f+1
    of the stream, so a block of rows is a contiguous range of pairs: a rank that owns
    some rows of a large batch generates only those."""
    assert 0 <= r0 <= r1 <= nrows
    f0, cnt = r0 * ncols, (r1 - r0) * ncols
    u = uniform(seed, 2 * f0, 2 * cnt)
    rad = np.sqrt(-2.0 * np.log(1.0 - u[0::2]))
    ang = 2.0 * np.pi * u[1::2]
    return (rad * np.cos(ang) + 1j * (rad * np.sin(ang))).reshape(r1 - r0, ncols)


# --------------------------------------------------------------------------------------
# Surfaces
# --------------------------------------------------------------------------------------

def fibonacci_sphere(n: int, radius: float = 1.0) -> np.ndarray:
    """Fibonacci lattice: z_i = 1-(2i+1)/n, phi_i = i*pi*(3-sqrt 5) mod 2pi.  [n,3] f64."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    ga = math.pi * (3.0 - math.sqrt(5.0))
    phi = np.mod(i * ga, 2.0 * math.pi)
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return radius * np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def _unit_directions(seed: int, start: int, count: int) -> np.ndarray:
    u = uniform(seed, 2 * start, 2 * count)
    z = 2.0 * u[0::2] - 1.0
    phi = 2.0 * math.pi * u[1::2]
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def spheroid_points(n: int, axes=(0.1, 0.1, 1.0), seed: int = 3) -> np.ndarray:
    """Area-uniform points on the ellipsoid x^2/a^2 + y^2/b^2 + z^2/c^2 = 1.

    A uniform sphere direction u maps to (a u_x, b u_y, c u_z); the ellipsoid's
    area element relative to the sphere's is a b c sqrt(sum u_i^2 / a_i^2), so the
    candidate is accepted with probability sqrt(sum u_i^2/a_i^2) / max_i(1/a_i).
    """
    a = np.asarray(axes, dtype=np.float64)
    inv_max = 1.0 / np.max(1.0 / a)
    out = []
    have = 0
    start = 0
    batch = max(1024, 2 * n)
    while have < n:
        d = _unit_directions(seed, start, batch)
        acc = uniform(seed + 0x5151, start, batch)
        p = np.sqrt(np.sum(d * d / (a * a), axis=1)) * inv_max
        keep = acc < p
        pts = d[keep] * a
        out.append(pts)
        have += pts.shape[0]
        start += batch
    return np.concatenate(out, axis=0)[:n]


CUBES = (((0.0, 0.0, 0.0), 20.0), ((10.0, 10.0, 10.0), 20.0), ((20.0, 20.0, 20.0), 20.0))


def cube_union_points(n: int, cubes=CUBES, seed: int = 4) -> np.ndarray:
    """Area-uniform points on the boundary of a union of axis-aligned cubes.

    Every cube face has the same area, so a candidate picks a cube and a face
    uniformly, a point uniformly on that face, and is rejected when it lies
    strictly inside another cube.
    """
    lo = np.array([c[0] for c in cubes], dtype=np.float64)
    side = np.array([c[1] for c in cubes], dtype=np.float64)
    nc = len(cubes)
    out = []
    have = 0
    start = 0
    batch = max(1024, 2 * n)
    while have < n:
        u = uniform(seed, 4 * start, 4 * batch).reshape(batch, 4)
        ci = np.minimum((u[:, 0] * nc).astype(np.int64), nc - 1)
        face = np.minimum((u[:, 1] * 6).astype(np.int64), 5)
        axis = face // 2
        high = face % 2
        s = side[ci]
        p = np.empty((batch, 3))
        # the two in-face coordinates
        a1 = (axis + 1) % 3
        a2 = (axis + 2) % 3
        rows = np.arange(batch)
        p[rows, axis] = lo[ci, axis] + high * s
        p[rows, a1] = lo[ci, a1] + u[:, 2] * s
        p[rows, a2] = lo[ci, a2] + u[:, 3] * s
        inside_other = np.zeros(batch, dtype=bool)
        for j in range(nc):
            strict = np.all((p > lo[j]) & (p < lo[j] + side[j]), axis=1)
            inside_other |= strict & (ci != j)
        pts = p[~inside_other]
        out.append(pts)
        have += pts.shape[0]
        start += batch
    return np.concatenate(out, axis=0)[:n]


def plane_wave_densities(points: np.ndarray, kappa: float, nrhs: int, seed: int, r0: int = 0,
                         r1: int | None = None) -> np.ndarray:
    """sigma_r(x) = A_r exp(i kappa d_r . x), d_r seeded unit vectors, A_r complex N(0,1).

    Returns complex128 [r1 - r0, N]: right-hand sides r0..r1-1 of the nrhs.
    """
    r1 = nrhs if r1 is None else r1
    d = _unit_directions(seed, r0, r1 - r0)
    amp = complex_normal(seed + 0x77, (nrhs,))[r0:r1]
    phase = kappa * (points @ d.T)  # [N, r1 - r0]
    return (amp[None, :] * np.exp(1j * phase)).T.copy()


def sample_targets(n: int, m: int, seed: int) -> np.ndarray:
    """First m entries of a seeded Fisher-Yates permutation of [0, n) (int64).

    Only the first m swaps are carried out, so the cost is O(m) for any n.
    """
    m = min(m, n)
    u = uniform(seed, 0, m)
    swaps: dict[int, int] = {}
    out = np.empty(m, dtype=np.int64)
    for i in range(m):
        j = min(i + int(u[i] * (n - i)), n - 1)
        vi = swaps.get(i, i)
        vj = swaps.get(j, j)
        swaps[i] = vj
        swaps[j] = vi
        out[i] = vj
    return out


DEGENERATE = ("two points", "line", "disc", "clusters")


def degenerate_points(kind: str):
    """Small degenerate point sets for edge-case checks: (points [n,3], kappa, levels).

    * "two points": two points in non-neighbouring leaves of a cube of side 0.3;
    * "line": 1200 collinear points along z (zero extent in x and y);
    * "disc": 1500 coplanar points on the unit disc z = 0;
    * "clusters": two Fibonacci spheres of radius 0.2 far apart (most boxes empty).
    """
    u = uniform(77, 0, 20000)
    if kind == "two points":
        return np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.1]]), 2 * math.pi, 3
    if kind == "line":
        z = np.sort(u[:1200]) * 2 - 1
        return np.stack([np.zeros(1200), np.zeros(1200), z], 1), 4 * math.pi, 5
    if kind == "disc":
        r, t = np.sqrt(u[:1500]), 2 * math.pi * u[1500:3000]
        return np.stack([r * np.cos(t), r * np.sin(t), np.zeros(1500)], 1), 4 * math.pi, 5
    if kind == "clusters":
        s = fibonacci_sphere(800) * 0.2
        return np.concatenate([s, s + np.array([3.0, 2.0, -1.0])]), 2 * math.pi, 6
    raise ValueError(kind)


# --------------------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------------------

@dataclass
class Workload:
    """One synthetic problem: points, wavenumber, tree/cone parameters, densities."""
    name: str
    n: int
    kappa: float
    levels: int
    p_radial: int = 3
    p_angular: int = 5
    leaf_ns: int = 1
    leaf_nc: int = 2
    nrhs: int = 1
    precision: str = "fp64"
    targets: int = 1000
    seed: int = 0
    surface: str = "sphere"
    leaf_max: int = 0
    description: str = ""
    _points: np.ndarray | None = field(default=None, repr=False)

    def points(self) -> np.ndarray:
        if self._points is None:
            if self.surface == "sphere":
                self._points = fibonacci_sphere(self.n)
            elif self.surface == "prolate":
                self._points = spheroid_points(self.n, (0.1, 0.1, 1.0), seed=self.seed)
            elif self.surface == "cubes":
                self._points = cube_union_points(self.n, seed=self.seed)
            elif self.surface == "random_sphere":
                d = _unit_directions(self.seed, 0, self.n)
                self._points = d
            else:
                raise ValueError(self.surface)
        return self._points

    def densities(self, rows=None) -> np.ndarray:
        """complex128 [nrhs, N]; rows = (r0, r1, batch) gives right-hand sides r0..r1-1 of
        a batch of `batch` right-hand sides drawn the same way (batch >= nrhs; the first
        nrhs rows of any batch are this workload's densities)."""
        r0, r1, batch = rows if rows is not None else (0, self.nrhs, self.nrhs)
        if self.surface == "cubes" and batch > 1:
            return plane_wave_densities(self.points(), self.kappa, batch, self.seed + 100, r0, r1)
        return complex_normal_rows(self.seed + 100, batch, self.n, r0, r1)

    def target_indices(self) -> np.ndarray:
        return sample_targets(self.n, self.targets, self.seed + 200)


def wavelengths_to_kappa(size: float, n_lambda: float) -> float:
    """kappa = 2 pi / lambda for a body of extent `size` spanning n_lambda wavelengths."""
    return 2.0 * math.pi * n_lambda / size


WORKLOADS = {
    # unit sphere, diameter 4 wavelengths, D = 4
    "sphere_4lambda": Workload("sphere_4lambda", 24_576, wavelengths_to_kappa(2.0, 4), 4,
                               leaf_ns=2, leaf_nc=4, targets=24_576, seed=1, surface="sphere",
                               description="Fibonacci sphere N=24576, 4 lambda, D=4, FP64"),
    # unit sphere, diameter 8 wavelengths, D = 6 (H_D = lambda/4, the paper's Sec. 4 setup)
    "sphere_8lambda": Workload("sphere_8lambda", 98_304, wavelengths_to_kappa(2.0, 8), 6,
                               leaf_ns=1, leaf_nc=2, targets=2_000, seed=6, surface="sphere",
                               description="Fibonacci sphere N=98304, 8 lambda, D=6, FP64"),
    # the same sphere with 16 right-hand sides on the tensor-core path (profiling size)
    "sphere_8lambda_16rhs": Workload("sphere_8lambda_16rhs", 98_304, wavelengths_to_kappa(2.0, 8), 6,
                                     leaf_ns=1, leaf_nc=2, nrhs=16, targets=1_000, seed=7, surface="sphere",
                                     precision="batched",
                                     description="Fibonacci sphere N=98304, 8 lambda, D=6, 16 RHS batched"),
    # unit sphere, diameter 32 wavelengths, D = 8
    "sphere_32lambda": Workload("sphere_32lambda", 393_216, wavelengths_to_kappa(2.0, 32), 8,
                                leaf_ns=1, leaf_nc=2, targets=2_000, seed=2, surface="sphere",
                                description="Fibonacci sphere N=393216, 32 lambda, D=8, FP64 + adjoint"),
    # higher order (P_s, P_ang) = (4, 7), 196 points per cone, for the 1e-5..1e-6 accuracy
    # range (the oracle gives 5.5e-5 with (1, 2) leaf cones and 3.6e-6 with (2, 4) on the
    # 8-wavelength sphere)
    "sphere_32lambda_p47": Workload("sphere_32lambda_p47", 393_216, wavelengths_to_kappa(2.0, 32), 8,
                                    p_radial=4, p_angular=7, leaf_ns=1, leaf_nc=2, targets=2_000, seed=2,
                                    surface="sphere",
                                    description="Fibonacci sphere N=393216, 32 lambda, D=8, order (4,7), FP64"),
    "sphere_8lambda_p47": Workload("sphere_8lambda_p47", 98_304, wavelengths_to_kappa(2.0, 8), 6,
                                   p_radial=4, p_angular=7, leaf_ns=2, leaf_nc=4, targets=2_000, seed=6,
                                   surface="sphere",
                                   description="Fibonacci sphere N=98304, 8 lambda, D=6, order (4,7), (2,4) leaf cones, FP64"),
    # prolate spheroid 10:1:1, long axis 128 wavelengths, D = 10
    "prolate_128lambda": Workload("prolate_128lambda", 3_145_728, wavelengths_to_kappa(2.0, 128), 10,
                                  leaf_ns=1, leaf_nc=2, targets=4_096, seed=3, surface="prolate",
                                  precision="mixed",
                                  description="prolate spheroid N=3145728, 128 lambda, D=10, mixed"),
    # the same spheroid on an adaptive octree of at most the same depth: boxes of level
    # >= 3 with at most 32 points are leaves (the cone sizes per level are those of the
    # uniform tree, whose leaf cones are chosen at level 10)
    "prolate_128lambda_adaptive": Workload("prolate_128lambda_adaptive", 3_145_728, wavelengths_to_kappa(2.0, 128),
                                           10, leaf_ns=1, leaf_nc=2, targets=4_096, seed=3, surface="prolate",
                                           precision="mixed", leaf_max=32,
                                           description="prolate spheroid N=3145728, 128 lambda, adaptive "
                                                       "octree (leaf_max 32, D <= 10), mixed"),
    # union of three cubes of side 20 wavelengths, 64 plane-wave RHS, D = 8
    "cubes_64rhs": Workload("cubes_64rhs", 1_572_864, 2.0 * math.pi, 8,
                            leaf_ns=1, leaf_nc=2, nrhs=64, targets=2_048, seed=4, surface="cubes",
                            precision="batched",
                            description="three-cube union N=1572864, lambda=1, 64 RHS"),
    # the three-cube union at 1/16 of the points with 6 levels and a quarter of the
    # wavenumber: leaf boxes of the same size in wavelengths and points per leaf as the
    # 8-level plan (profiling size for the tensor-core cone kernel)
    "cubes_98k_64rhs": Workload("cubes_98k_64rhs", 98_304, 2.0 * math.pi / 4.0, 6,
                                leaf_ns=1, leaf_nc=2, nrhs=64, targets=512, seed=4, surface="cubes",
                                precision="batched",
                                description="three-cube union N=98304, 64 RHS (profiling size)"),
    # Laplace kernel (kappa = 0) on the unit sphere, N = 6,291,456 (the largest sphere of
    # the paper's Laplace table), D = 8 (about 82 points per leaf box); a fixed number of
    # cone segments per box at every level, (n_s, n_C) = (3, 6)
    "sphere_laplace_6M": Workload("sphere_laplace_6M", 6_291_456, 0.0, 8, leaf_ns=3, leaf_nc=6,
                                  targets=1_000, seed=8, surface="sphere", precision="mixed",
                                  description="Fibonacci sphere N=6291456, Laplace (kappa=0), D=8, mixed"),
    # unit sphere, diameter 256 wavelengths, D = 9, 8 RHS
    "sphere_256lambda": Workload("sphere_256lambda", 25_165_824, wavelengths_to_kappa(2.0, 256), 9,
                                 leaf_ns=3, leaf_nc=6, nrhs=8, targets=1_024, seed=5, surface="sphere",
                                 precision="mixed",
                                 description="Fibonacci sphere N=25165824, 256 lambda, D=9, 8 RHS"),
    # the 256-wavelength sphere scaled down 16x (same leaf box width of one wavelength,
    # same leaf cones, same points per leaf): its kernels see the same per-box geometry
    # with level arrays of about 1 GB, so single kernels of it can be profiled
    "sphere_64lambda": Workload("sphere_64lambda", 1_572_864, wavelengths_to_kappa(2.0, 64), 7,
                                leaf_ns=3, leaf_nc=6, nrhs=8, targets=1_024, seed=5, surface="sphere",
                                precision="mixed",
                                description="Fibonacci sphere N=1572864, 64 lambda, D=7, 8 RHS"),
}


def small_sphere(n: int, n_lambda: float, levels: int, leaf_ns=1, leaf_nc=2, seed=11,
                 nrhs=1) -> Workload:
    """A small Fibonacci-sphere case sized for the oracle (test use)."""
    return Workload(f"sphere_n{n}", n, wavelengths_to_kappa(2.0, n_lambda), levels,
                    leaf_ns=leaf_ns, leaf_nc=leaf_nc, nrhs=nrhs, targets=n, seed=seed,
                    surface="sphere")
