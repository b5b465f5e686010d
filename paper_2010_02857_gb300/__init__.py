"""GB300 (sm_103a) implementation of the IFGF method (Bauinger & Bruno, arXiv 2010.02857).

Python binding of the C ABI declared in include/ifgf.h.  Every entry point here
only marshals arguments (torch tensors or numpy arrays -> pointers, sizes and the
current CUDA stream) and calls libifgf.so; all computation runs in the library's
CUDA kernels.  There is no CPU fallback: importing works without the library, but
every call raises if libifgf.so has not been built.

    plan_create(points, kappa, levels, p_radial=3, p_angular=5, ...) -> handle
    apply(handle, sigma, u, nrhs)          u = A sigma        (Eq. field1)
    apply_adjoint(handle, v, w, nrhs)      w = A^H v
    plan_destroy(handle)

`Plan` wraps a handle; `IFGFApply` is a torch.autograd.Function whose backward is
the library's hand-written adjoint.  rhs_shard / apply_rhs_sharded split a batch of
right-hand sides over ranks (one GPU and one plan per rank, no data-path collective).
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libifgf.so")

IFGF_FP64, IFGF_MIXED, IFGF_BATCHED_BF16, IFGF_BATCHED_FP16 = 0, 1, 2, 3
PRECISIONS = {"fp64": IFGF_FP64, "mixed": IFGF_MIXED, "batched": IFGF_BATCHED_BF16,
              "batched_bf16": IFGF_BATCHED_BF16, "batched_fp16": IFGF_BATCHED_FP16}
STATUS = {0: "IFGF_OK", 1: "IFGF_EINVAL", 2: "IFGF_ENOMEM", 3: "IFGF_ECUDA", 4: "IFGF_ETIMEOUT",
          5: "IFGF_EINTERNAL"}

# every symbol include/ifgf.h declares
EXPORTS = ["ifgf_plan_create", "ifgf_apply", "ifgf_apply_adjoint", "ifgf_apply_partial", "ifgf_apply_noalloc",
           "ifgf_plan_destroy", "ifgf_plan_level_info", "ifgf_plan_get_perm", "ifgf_plan_get_boxes",
           "ifgf_plan_get_box_ends", "ifgf_plan_get_point_levels", "ifgf_plan_get_near",
           "ifgf_plan_get_cousins", "ifgf_plan_get_active", "ifgf_plan_get_values", "ifgf_plan_cone_ids",
           "ifgf_plan_geometry",
           "ifgf_plan_stats", "ifgf_plan_check", "ifgf_plan_set_profiling", "ifgf_plan_set_graphs", "ifgf_plan_autotune", "ifgf_plan_set_tiles", "ifgf_plan_timings",
           "ifgf_plan_tune_key", "ifgf_tune_cache_lookup", "ifgf_tune_cache_store", "ifgf_plan_autotune_cached",
           "ifgf_device_peak", "ifgf_last_error"]
STAGES = ["permute_in", "leaf", "upward", "eval", "permute_out", "adj_level", "adj_eval", "adj_lists"]
LEAF_SHAPES = ["16x8", "32x4", "8x16"]


class IFGFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class ifgf_options(ctypes.Structure):
    _fields_ = [("leaf_ns", ctypes.c_int), ("leaf_nc", ctypes.c_int), ("max_nrhs", ctypes.c_int),
                ("precision", ctypes.c_int), ("flags", ctypes.c_int), ("value_budget_bytes", ctypes.c_longlong),
                ("timeout_s", ctypes.c_double), ("leaf_max", ctypes.c_int)]


_lib = None


def lib():
    """Load libifgf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libifgf.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.ifgf_plan_create.argtypes = [P, i64, d, i, i, i, ctypes.POINTER(ifgf_options), P, ctypes.POINTER(P)]
        L.ifgf_apply.argtypes = [P, P, P, i, P]
        L.ifgf_apply_adjoint.argtypes = [P, P, P, i, P]
        L.ifgf_apply_partial.argtypes = [P, P, P, i, i, i, P]
        L.ifgf_apply_noalloc.argtypes = [P, P, P, i, P]
        L.ifgf_plan_destroy.argtypes = [P]
        L.ifgf_plan_level_info.argtypes = [P, i, P]
        L.ifgf_plan_get_perm.argtypes = [P, P]
        L.ifgf_plan_get_boxes.argtypes = [P, i, P, P]
        L.ifgf_plan_get_cousins.argtypes = [P, i, P, P]
        L.ifgf_plan_get_box_ends.argtypes = [P, i, P, P]
        L.ifgf_plan_get_point_levels.argtypes = [P, P]
        L.ifgf_plan_get_near.argtypes = [P, i, P, P, P, P]
        L.ifgf_plan_get_active.argtypes = [P, i, P, P]
        L.ifgf_plan_get_values.argtypes = [P, i, P]
        L.ifgf_plan_cone_ids.argtypes = [P, i, i64, P, P, P]
        L.ifgf_plan_geometry.argtypes = [P, P]
        L.ifgf_plan_stats.argtypes = [P, ctypes.c_char_p, ctypes.c_size_t]
        L.ifgf_plan_check.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
        L.ifgf_plan_set_profiling.argtypes = [P, i]
        L.ifgf_plan_set_graphs.argtypes = [P, i]
        L.ifgf_plan_autotune.argtypes = [P, i, i, P, P, P]
        L.ifgf_plan_set_tiles.argtypes = [P, i, i]
        L.ifgf_plan_tune_key.argtypes = [P, i, ctypes.c_char_p, i]
        L.ifgf_tune_cache_lookup.argtypes = [ctypes.c_char_p, ctypes.c_char_p, P, P]
        L.ifgf_tune_cache_store.argtypes = [ctypes.c_char_p, ctypes.c_char_p, P]
        L.ifgf_plan_autotune_cached.argtypes = [P, i, i, ctypes.c_char_p, P, P, P]
        L.ifgf_plan_timings.argtypes = [P, P, P, P, i]
        L.ifgf_device_peak.argtypes = [i, P, P]
        L.ifgf_last_error.argtypes = [P]
        L.ifgf_last_error.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name != "ifgf_last_error":
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status: int, handle=None):
    if status != 0:
        msg = lib().ifgf_last_error(handle)
        raise IFGFError(status, msg.decode() if msg else "")


def _ptr(x):
    """Pointer of a torch tensor or numpy array (must be contiguous)."""
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return ctypes.c_void_p(x.ctypes.data)
    assert x.is_contiguous()
    return ctypes.c_void_p(x.data_ptr())


def _stream(x=None):
    try:
        import torch
        if x is not None and hasattr(x, "is_cuda") and x.is_cuda:
            return ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


# ------------------------------------------------------------------------------------
# C-ABI mirrors
# ------------------------------------------------------------------------------------

def plan_create(points, kappa: float, levels: int, p_radial: int = 3, p_angular: int = 5,
                leaf_ns: int = 0, leaf_nc: int = 0, max_nrhs: int = 1, precision="fp64",
                flags: int = 0, value_budget_bytes: int = 0, timeout_s: float = 0.0, stream=None,
                leaf_max: int = 0):
    """ifgf_plan_create; points: [N,3] float64 (numpy or torch, host or device); leaf_max > 0
    builds an adaptive octree."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    if isinstance(points, np.ndarray):
        points = np.ascontiguousarray(points, dtype=np.float64)
        n = points.shape[0]
    else:
        points = points.contiguous()
        n = points.shape[0]
    opt = ifgf_options(int(leaf_ns), int(leaf_nc), int(max_nrhs), int(precision), int(flags),
                       int(value_budget_bytes), float(timeout_s), int(leaf_max))
    h = ctypes.c_void_p()
    st = stream if stream is not None else _stream(points)
    _check(lib().ifgf_plan_create(_ptr(points), n, float(kappa), int(levels), int(p_radial),
                                  int(p_angular), ctypes.byref(opt), st, ctypes.byref(h)))
    return h


def apply(handle, sigma, u, nrhs: int, stream=None):
    _check(lib().ifgf_apply(handle, _ptr(sigma), _ptr(u), int(nrhs),
                            stream if stream is not None else _stream(sigma)), handle)


def apply_adjoint(handle, v, w, nrhs: int, stream=None):
    _check(lib().ifgf_apply_adjoint(handle, _ptr(v), _ptr(w), int(nrhs),
                                    stream if stream is not None else _stream(v)), handle)


def apply_partial(handle, x, y, nrhs: int, mode: int, adjoint: bool = False, stream=None):
    _check(lib().ifgf_apply_partial(handle, _ptr(x), _ptr(y), int(nrhs), int(mode), int(bool(adjoint)),
                                    stream if stream is not None else _stream(x)), handle)


def apply_noalloc(handle, sigma, u, nrhs: int, stream=None):
    """ifgf_apply_noalloc: like apply(), with all scratch in the library's fixed 64 MiB
    device array (device tensors only; the library allocates nothing)."""
    _check(lib().ifgf_apply_noalloc(handle, _ptr(sigma), _ptr(u), int(nrhs),
                                    stream if stream is not None else _stream(sigma)), handle)


def device_peak(which: str, stream=None) -> float:
    """ifgf_device_peak: the current device's measured FMA rate in TFLOP/s, which =
    "fp64" or "fp32" (a roofline denominator)."""
    out = ctypes.c_double(0.0)
    _check(lib().ifgf_device_peak({"fp64": 0, "fp32": 1}[which], ctypes.byref(out),
                                  stream if stream is not None else _stream()))
    return float(out.value)


def plan_destroy(handle):
    _check(lib().ifgf_plan_destroy(handle))


def tune_cache_lookup(path: str, key: str):
    """ifgf_tune_cache_lookup: (leaf_shape, cone_ctas_per_sm) stored for key in the tune
    cache file, or None."""
    found = ctypes.c_int(0)
    choice = (ctypes.c_int * 2)()
    _check(lib().ifgf_tune_cache_lookup(os.fsencode(path), key.encode(), ctypes.byref(found), choice))
    return (int(choice[0]), int(choice[1])) if found.value else None


def tune_cache_store(path: str, key: str, leaf_shape: int, cone_ctas_per_sm: int):
    """ifgf_tune_cache_store: append a tile-shape choice for key to the tune cache file."""
    choice = (ctypes.c_int * 2)(int(leaf_shape), int(cone_ctas_per_sm))
    _check(lib().ifgf_tune_cache_store(os.fsencode(path), key.encode(), choice))


# ------------------------------------------------------------------------------------
# Object wrapper
# ------------------------------------------------------------------------------------

class Plan:
    """An IFGF plan on the current CUDA device."""

    def __init__(self, points, kappa, levels, p_radial=3, p_angular=5, leaf_ns=0, leaf_nc=0,
                 max_nrhs=1, precision="fp64", flags=0, value_budget_bytes=0, timeout_s=0.0, leaf_max=0):
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.n = int(points.shape[0])
        self.levels = int(levels)
        self.max_nrhs = int(max_nrhs)
        self.P = p_radial * p_angular * p_angular
        self.handle = plan_create(points, kappa, levels, p_radial, p_angular, leaf_ns, leaf_nc,
                                  max_nrhs, self.precision, flags, value_budget_bytes, timeout_s,
                                  leaf_max=leaf_max)

    @property
    def complex_dtype(self):
        import torch
        return torch.complex128 if self.precision == IFGF_FP64 else torch.complex64

    @property
    def numpy_dtype(self):
        return np.complex128 if self.precision == IFGF_FP64 else np.complex64

    def close(self):
        if getattr(self, "handle", None):
            plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _out_like(self, x):
        if isinstance(x, np.ndarray):
            return np.empty_like(x)
        import torch
        return torch.empty_like(x)

    def _prep(self, x):
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=self.numpy_dtype)
            if x.ndim == 1:
                x = x[None, :]
        else:
            x = x.to(self.complex_dtype).contiguous()
            if x.dim() == 1:
                x = x[None, :]
        assert x.shape[1] == self.n
        return x

    def apply(self, sigma, out=None):
        sigma = self._prep(sigma)
        u = self._out_like(sigma) if out is None else out
        apply(self.handle, sigma, u, sigma.shape[0])
        return u

    def apply_adjoint(self, v, out=None):
        v = self._prep(v)
        w = self._out_like(v) if out is None else out
        apply_adjoint(self.handle, v, w, v.shape[0])
        return w

    def apply_partial(self, x, mode, adjoint=False):
        x = self._prep(x)
        y = self._out_like(x)
        apply_partial(self.handle, x, y, x.shape[0], mode, adjoint)
        return y

    # introspection
    def level_info(self, d):
        v = np.zeros(8, dtype=np.int64)
        _check(lib().ifgf_plan_level_info(self.handle, d, _ptr(v)), self.handle)
        keys = ["nbox", "nnbr", "ncous", "nact", "ns", "nc", "cousin_evals", "upward_evals"]
        return {k: int(x) for k, x in zip(keys, v)}

    def perm(self):
        out = np.zeros(self.n, dtype=np.int64)
        _check(lib().ifgf_plan_get_perm(self.handle, _ptr(out)), self.handle)
        return out

    def boxes(self, d):
        nb = self.level_info(d)["nbox"]
        keys = np.zeros(nb, dtype=np.uint64)
        start = np.zeros(nb + 1, dtype=np.int64)
        _check(lib().ifgf_plan_get_boxes(self.handle, d, _ptr(keys), _ptr(start)), self.handle)
        return keys, start

    def box_ends(self, d):
        """(end, leaf) of the boxes of level d (see ifgf_plan_get_box_ends)."""
        nb = self.level_info(d)["nbox"]
        end = np.zeros(max(nb, 1), dtype=np.int64)
        leaf = np.zeros(max(nb, 1), dtype=np.int64)
        _check(lib().ifgf_plan_get_box_ends(self.handle, d, _ptr(end), _ptr(leaf)), self.handle)
        return end[:nb], leaf[:nb].astype(bool)

    def point_levels(self):
        out = np.zeros(self.n, dtype=np.int64)
        _check(lib().ifgf_plan_get_point_levels(self.handle, _ptr(out)), self.handle)
        return out

    def near(self, d):
        """Near-field ranges of the leaf boxes of level d: (start, lo, hi)."""
        m = ctypes.c_int64(0)
        _check(lib().ifgf_plan_get_near(self.handle, d, ctypes.byref(m), None, None, None), self.handle)
        nb = self.level_info(d)["nbox"]
        start = np.zeros(nb + 1, dtype=np.int64)
        lo = np.zeros(max(m.value, 1), dtype=np.int64)
        hi = np.zeros(max(m.value, 1), dtype=np.int64)
        _check(lib().ifgf_plan_get_near(self.handle, d, ctypes.byref(m), _ptr(start), _ptr(lo), _ptr(hi)),
               self.handle)
        return start, lo[: m.value], hi[: m.value]

    def cousins(self, d):
        li = self.level_info(d)
        start = np.zeros(li["nbox"] + 1, dtype=np.int64)
        lst = np.zeros(max(li["ncous"], 1), dtype=np.int64)
        _check(lib().ifgf_plan_get_cousins(self.handle, d, _ptr(start), _ptr(lst)), self.handle)
        return start, lst[: li["ncous"]]

    def active(self, d):
        li = self.level_info(d)
        start = np.zeros(li["nbox"] + 1, dtype=np.int64)
        cones = np.zeros(max(li["nact"], 1), dtype=np.int64)
        _check(lib().ifgf_plan_get_active(self.handle, d, _ptr(start), _ptr(cones)), self.handle)
        return start, cones[: li["nact"]]

    def values(self, d, nrhs=1):
        li = self.level_info(d)
        out = np.zeros((li["nact"], self.P, nrhs), dtype=self.numpy_dtype)
        _check(lib().ifgf_plan_get_values(self.handle, d, _ptr(out)), self.handle)
        return out

    def cone_ids(self, d, v):
        """Cone ids of the vectors v [n,3] at level d: (exact path, fast path)."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        ex = np.zeros(v.shape[0], dtype=np.int32)
        fa = np.zeros(v.shape[0], dtype=np.int32)
        _check(lib().ifgf_plan_cone_ids(self.handle, d, v.shape[0], _ptr(v), _ptr(ex), _ptr(fa)), self.handle)
        return ex, fa

    def geometry(self):
        g = np.zeros(4)
        _check(lib().ifgf_plan_geometry(self.handle, _ptr(g)), self.handle)
        return g[0], g[1:].copy()

    def stats(self):
        buf = ctypes.create_string_buffer(1 << 16)
        _check(lib().ifgf_plan_stats(self.handle, buf, len(buf)), self.handle)
        return json.loads(buf.value.decode())

    def set_profiling(self, on: bool):
        _check(lib().ifgf_plan_set_profiling(self.handle, int(bool(on))), self.handle)

    def autotune(self, nrhs: int, reps: int = 3, cache: str | None = None) -> dict:
        """Time the batched path's tile shapes on this plan and keep the fastest.

        With ``cache`` (a file path), a shape choice stored there for this plan's key is
        taken without timing (``"cached": True``), and a new choice is appended to it.
        """
        choice = np.zeros(2, dtype=np.int32)
        if cache is not None:
            hit = np.zeros(1, dtype=np.int32)
            _check(lib().ifgf_plan_autotune_cached(self.handle, int(nrhs), int(reps), os.fsencode(cache),
                                                   _ptr(choice), _ptr(hit), _stream()), self.handle)
            return {"leaf_shape": LEAF_SHAPES[int(choice[0])], "cone_ctas_per_sm": int(choice[1]),
                    "cached": bool(hit[0]), "key": self.tune_key(nrhs)}
        ms = np.zeros(5)
        _check(lib().ifgf_plan_autotune(self.handle, int(nrhs), int(reps), _ptr(ms), _ptr(choice), _stream()),
               self.handle)
        return {"leaf_shape": LEAF_SHAPES[int(choice[0])], "cone_ctas_per_sm": int(choice[1]),
                "leaf_ms": [float(x) for x in ms[:3]], "cone_ms": [float(x) for x in ms[3:]]}

    def tune_key(self, nrhs: int) -> str:
        """The tune-cache key of this plan for nrhs right-hand sides."""
        buf = ctypes.create_string_buffer(512)
        _check(lib().ifgf_plan_tune_key(self.handle, int(nrhs), buf, len(buf)), self.handle)
        return buf.value.decode()

    def set_tiles(self, leaf_shape: int, cone_ctas_per_sm: int):
        """Set the batched path's tile shapes (leaf shape 0..2, 1 or 2 CTAs per SM)."""
        _check(lib().ifgf_plan_set_tiles(self.handle, int(leaf_shape), int(cone_ctas_per_sm)), self.handle)

    def set_graphs(self, on: bool):
        """Capture each evaluation into a CUDA graph on first use and replay it after."""
        _check(lib().ifgf_plan_set_graphs(self.handle, int(bool(on))), self.handle)

    def timings(self) -> dict:
        ms = np.zeros(len(STAGES))
        launches = np.zeros(len(STAGES), dtype=np.int64)
        calls = np.zeros(1, dtype=np.int64)
        _check(lib().ifgf_plan_timings(self.handle, _ptr(ms), _ptr(launches), _ptr(calls), len(STAGES)),
               self.handle)
        return {"calls": int(calls[0]),
                "stages": {s: {"ms": float(m), "launches": int(l)} for s, m, l in zip(STAGES, ms, launches)}}

    def check(self) -> int:
        e = ctypes.c_int(0)
        _check(lib().ifgf_plan_check(self.handle, ctypes.byref(e)), self.handle)
        return int(e.value)


# ------------------------------------------------------------------------------------
# Right-hand sides sharded over ranks (one GPU per rank)
# ------------------------------------------------------------------------------------

def rhs_shard(nrhs: int, rank: int, world: int) -> tuple[int, int]:
    """The right-hand sides [r0, r1) of `rank` when a batch of nrhs is split over `world`
    ranks: contiguous rows of the [nrhs][N] batch, sizes differing by at most one, in rank
    order.  Right-hand sides are independent problems of the same operator, so every rank
    applies its own plan (a replica of the same geometry on its own GPU) to its rows and
    no data crosses ranks while they evaluate."""
    if world < 1 or not 0 <= rank < world or nrhs < 0:
        raise ValueError("need 0 <= rank < world and nrhs >= 0")
    base, extra = divmod(nrhs, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def apply_rhs_sharded(plan: "Plan", sigma_batch, rank: int, world: int, adjoint: bool = False):
    """This rank's rows of A sigma (or A^H sigma) for a [nrhs][N] batch: the rows
    rhs_shard(nrhs, rank, world) of sigma_batch, applied on this rank's plan.  Returns
    ((r0, r1), u_rows); a rank with no rows returns an empty [0][N] array."""
    r0, r1 = rhs_shard(int(sigma_batch.shape[0]), rank, world)
    rows = sigma_batch[r0:r1]
    if r1 == r0:
        return (r0, r1), rows
    return (r0, r1), (plan.apply_adjoint(rows) if adjoint else plan.apply(rows))


def gather_rhs_shards(u_rows, nrhs: int, group=None):
    """Reassembles the [nrhs][N] result from every rank's rows (torch.distributed
    all_gather on the host; for callers that need the whole batch on every rank, outside
    any timed evaluation).  u_rows: this rank's rows as a numpy array."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    shards = [rhs_shard(nrhs, r, world) for r in range(world)]
    rows = max(b - a for a, b in shards)  # every rank sends the same shape (padded)
    mine = np.ascontiguousarray(u_rows)
    buf = np.zeros((rows, mine.shape[1]), dtype=mine.dtype)
    buf[: mine.shape[0]] = mine
    send = torch.from_numpy(buf)
    parts = [torch.empty_like(send) for _ in range(world)]
    dist.all_gather(parts, send, group=group)
    return np.concatenate([p.numpy()[: b - a] for p, (a, b) in zip(parts, shards)], axis=0)


def _autograd_function():
    import torch

    class IFGFApply(torch.autograd.Function):
        """u = A sigma with backward grad_sigma = A^H grad_u (PyTorch's conjugate-Wirtinger
        convention for a C-linear map), both through the library's kernels."""

        @staticmethod
        def forward(ctx, sigma, plan):
            ctx.plan = plan
            return plan.apply(sigma)

        @staticmethod
        def backward(ctx, grad_u):
            return ctx.plan.apply_adjoint(grad_u.contiguous()), None

    return IFGFApply


_IFGFApply = None


def ifgf_apply_autograd(sigma, plan):
    """Differentiable u = A sigma (torch tensors on the plan's device)."""
    global _IFGFApply
    if _IFGFApply is None:
        _IFGFApply = _autograd_function()
    return _IFGFApply.apply(sigma, plan)
