"""CPU FP64 oracle for the IFGF method (test infrastructure only).

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg may import this module.  The GPU library never calls it.

`build()` compiles ifgf_oracle.c with gcc (-O2 -ffp-contract=off -fopenmp) into
oracle/_build/liboracle.so; the classes below marshal numpy arrays to it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ifgf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or older than its source."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            d = ctypes.c_double
            i = ctypes.c_int
            L.oracle_direct.argtypes = [i64, P, d, i, P, i64, P, P]
            L.oracle_direct_adjoint.argtypes = [i64, P, d, i, P, i64, P, P]
            L.oracle_plan_create.argtypes = [i64, P, d, i, i, i, i, i]
            L.oracle_plan_create.restype = P
            L.oracle_plan_create_adaptive.argtypes = [i64, P, d, i, i, i, i, i, i64]
            L.oracle_plan_create_adaptive.restype = P
            L.oracle_get_box_ends.argtypes = [P, i, P, P]
            L.oracle_get_near.argtypes = [P, i, P, P, P]
            L.oracle_get_near.restype = i64
            L.oracle_get_point_levels.argtypes = [P, P]
            L.oracle_plan_destroy.argtypes = [P]
            L.oracle_apply.argtypes = [P, i, P, P, i]
            L.oracle_apply_adjoint.argtypes = [P, i, P, P, i]
            L.oracle_plan_info.argtypes = [P, P]
            L.oracle_plan_geometry.argtypes = [P, P]
            L.oracle_level_info.argtypes = [P, i, P]
            L.oracle_level_params.argtypes = [P, i, P]
            L.oracle_get_perm.argtypes = [P, P]
            L.oracle_get_boxes.argtypes = [P, i, P, P]
            L.oracle_get_neighbors.argtypes = [P, i, P, P]
            L.oracle_get_cousins.argtypes = [P, i, P, P]
            L.oracle_get_active.argtypes = [P, i, P, P]
            L.oracle_get_F.argtypes = [P, i, P]
            L.oracle_cone_of.argtypes = [P, i, P, P, P, P]
            L.oracle_node_pos.argtypes = [P, i, i64, i, P, P]
            L.oracle_node_pos.restype = d
            L.oracle_box_center.argtypes = [P, i, ctypes.c_uint64, P]
            L.oracle_node_rel_child.argtypes = [P, i, i64, i, i, P]
            L.oracle_green.argtypes = [P, P, d, P]
            L.oracle_analytic_factor.argtypes = [P, P, P, d, P]
            L.oracle_cheb_nodes.argtypes = [i, P]
            L.oracle_lagrange.argtypes = [i, d, P]
            L.oracle_num_threads.restype = i
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _as_c128(a, n) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    if a.ndim == 1:
        a = a[None, :]
    assert a.shape[1] == n
    return a


def direct(points, kappa, sigma, targets=None) -> np.ndarray:
    """Exact sum of Eq. (field1) at the listed targets.  sigma: [nrhs, N] -> [nrhs, M]."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n = pts.shape[0]
    s = _as_c128(sigma, n)
    t = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    out = np.zeros((s.shape[0], t.shape[0]), dtype=np.complex128)
    lib().oracle_direct(n, _p(pts), float(kappa), s.shape[0], _p(s), t.shape[0], _p(t), _p(out))
    return out


def direct_adjoint(points, kappa, v, sources=None) -> np.ndarray:
    """Conjugate transpose of Eq. (field1) at the listed source indices."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n = pts.shape[0]
    s = _as_c128(v, n)
    t = np.arange(n, dtype=np.int64) if sources is None else np.ascontiguousarray(sources, dtype=np.int64)
    out = np.zeros((s.shape[0], t.shape[0]), dtype=np.complex128)
    lib().oracle_direct_adjoint(n, _p(pts), float(kappa), s.shape[0], _p(s), t.shape[0], _p(t), _p(out))
    return out


def green(x, y, kappa) -> complex:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.zeros(2)
    lib().oracle_green(_p(x), _p(y), float(kappa), _p(out))
    return complex(out[0], out[1])


def analytic_factor(x, xs, xp, kappa) -> complex:
    x = np.ascontiguousarray(x, dtype=np.float64)
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    xp = np.ascontiguousarray(xp, dtype=np.float64)
    out = np.zeros(2)
    lib().oracle_analytic_factor(_p(x), _p(xs), _p(xp), float(kappa), _p(out))
    return complex(out[0], out[1])


def cheb_nodes(n: int) -> np.ndarray:
    out = np.zeros(n)
    lib().oracle_cheb_nodes(n, _p(out))
    return out


def lagrange(n: int, t: float) -> np.ndarray:
    out = np.zeros(n)
    lib().oracle_lagrange(n, float(t), _p(out))
    return out


def num_threads() -> int:
    return lib().oracle_num_threads()


class Plan:
    """Serial CPU IFGF (Algorithm 1) on a fixed point set."""

    def __init__(self, points, kappa, levels, p_radial=3, p_angular=5, leaf_ns=1, leaf_nc=2, leaf_max=0):
        """leaf_max > 0 builds the adaptive octree (a box of level >= 3 with at most
        leaf_max points is a leaf); 0 the uniform one of `levels` levels."""
        self.points = np.ascontiguousarray(points, dtype=np.float64)
        self.n = self.points.shape[0]
        self.kappa = float(kappa)
        self.levels = int(levels)
        self.leaf_max = int(leaf_max)
        self.h = lib().oracle_plan_create_adaptive(self.n, _p(self.points), self.kappa, self.levels,
                                                   int(p_radial), int(p_angular), int(leaf_ns), int(leaf_nc),
                                                   self.leaf_max)
        if not self.h:
            raise ValueError("oracle_plan_create rejected the input")
        info = np.zeros(6, dtype=np.int64)
        lib().oracle_plan_info(self.h, _p(info))
        self.P = int(info[2])

    def close(self):
        if getattr(self, "h", None):
            lib().oracle_plan_destroy(self.h)
            self.h = None

    __del__ = close

    def apply(self, sigma, mode: int = 3) -> np.ndarray:
        s = _as_c128(sigma, self.n)
        u = np.zeros_like(s)
        rc = lib().oracle_apply(self.h, s.shape[0], _p(s), _p(u), int(mode))
        if rc != 0:
            raise RuntimeError("oracle IFGF: a target or node fell in a non-relevant cone")
        return u

    def apply_adjoint(self, v, mode: int = 3) -> np.ndarray:
        s = _as_c128(v, self.n)
        w = np.zeros_like(s)
        rc = lib().oracle_apply_adjoint(self.h, s.shape[0], _p(s), _p(w), int(mode))
        if rc != 0:
            raise RuntimeError("oracle IFGF adjoint: missing relevant cone")
        return w

    def info(self) -> dict:
        info = np.zeros(6, dtype=np.int64)
        lib().oracle_plan_info(self.h, _p(info))
        return dict(n=int(info[0]), levels=int(info[1]), P=int(info[2]), near_pairs=int(info[5]))

    def geometry(self):
        g = np.zeros(4)
        lib().oracle_plan_geometry(self.h, _p(g))
        return g[0], g[1:].copy()

    def level_info(self, d: int) -> dict:
        v = np.zeros(8, dtype=np.int64)
        lib().oracle_level_info(self.h, d, _p(v))
        keys = ["nbox", "nnbr", "ncous", "nact", "ns", "nc", "cousin_evals", "upward_evals"]
        return {k: int(x) for k, x in zip(keys, v)}

    def level_params(self, d: int) -> dict:
        v = np.zeros(4)
        lib().oracle_level_params(self.h, d, _p(v))
        return dict(H=v[0], h=v[1], ds=v[2], dth=v[3])

    def perm(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.int64)
        lib().oracle_get_perm(self.h, _p(out))
        return out

    def boxes(self, d: int):
        nb = self.level_info(d)["nbox"]
        keys = np.zeros(nb, dtype=np.uint64)
        start = np.zeros(nb + 1, dtype=np.int64)
        lib().oracle_get_boxes(self.h, d, _p(keys), _p(start))
        return keys, start

    def box_ends(self, d: int):
        """(end, leaf) of the boxes of level d: box b holds the sorted points
        start[b] .. end[b] - 1; leaf boxes are not subdivided."""
        nb = self.level_info(d)["nbox"]
        end = np.zeros(nb, dtype=np.int64)
        leaf = np.zeros(nb, dtype=np.int64)
        lib().oracle_get_box_ends(self.h, d, _p(end), _p(leaf))
        return end, leaf.astype(bool)

    def near(self, d: int):
        """Near-field point ranges of the leaf boxes of level d >= 3: (start, lo, hi)."""
        m = lib().oracle_get_near(self.h, d, None, None, None)
        nb = self.level_info(d)["nbox"]
        start = np.zeros(nb + 1, dtype=np.int64)
        lo = np.zeros(max(m, 1), dtype=np.int64)
        hi = np.zeros(max(m, 1), dtype=np.int64)
        lib().oracle_get_near(self.h, d, _p(start), _p(lo), _p(hi))
        return start, lo[:m], hi[:m]

    def point_levels(self):
        """Leaf level of every point, in sorted (Morton) order."""
        out = np.zeros(self.n, dtype=np.int64)
        lib().oracle_get_point_levels(self.h, _p(out))
        return out

    def neighbors(self, d: int):
        li = self.level_info(d)
        start = np.zeros(li["nbox"] + 1, dtype=np.int64)
        lst = np.zeros(max(li["nnbr"], 1), dtype=np.int64)
        lib().oracle_get_neighbors(self.h, d, _p(start), _p(lst))
        return start, lst[: li["nnbr"]]

    def cousins(self, d: int):
        li = self.level_info(d)
        start = np.zeros(li["nbox"] + 1, dtype=np.int64)
        lst = np.zeros(max(li["ncous"], 1), dtype=np.int64)
        lib().oracle_get_cousins(self.h, d, _p(start), _p(lst))
        return start, lst[: li["ncous"]]

    def active(self, d: int):
        li = self.level_info(d)
        start = np.zeros(li["nbox"] + 1, dtype=np.int64)
        cones = np.zeros(max(li["nact"], 1), dtype=np.int64)
        lib().oracle_get_active(self.h, d, _p(start), _p(cones))
        return start, cones[: li["nact"]]

    def F(self, d: int, nrhs: int = 1) -> np.ndarray:
        li = self.level_info(d)
        out = np.zeros((li["nact"], self.P, nrhs), dtype=np.complex128)
        lib().oracle_get_F(self.h, d, _p(out))
        return out

    def cone_of(self, d: int, y, c):
        y = np.ascontiguousarray(y, dtype=np.float64)
        c = np.ascontiguousarray(c, dtype=np.float64)
        g = np.zeros(4, dtype=np.int64)
        loc = np.zeros(3)
        lib().oracle_cone_of(self.h, d, _p(y), _p(c), _p(g), _p(loc))
        return g, loc

    def node_pos(self, d: int, cone: int, node: int, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        q = np.zeros(3)
        R = lib().oracle_node_pos(self.h, d, int(cone), int(node), _p(x), _p(q))
        return q, R

    def node_rel_child(self, d: int, cone: int, node: int, octant: int):
        """Interpolation point of a level-(d-1) parent cone relative to the centre of the
        child (level d) in the given octant."""
        v = np.zeros(3)
        lib().oracle_node_rel_child(self.h, d, int(cone), int(node), int(octant), _p(v))
        return v

    def box_center(self, d: int, key: int):
        c = np.zeros(3)
        lib().oracle_box_center(self.h, d, int(key), _p(c))
        return c
