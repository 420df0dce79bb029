"""Python binding of libdipole (include/dipole.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module checks
tensor devices, dtypes and shapes, passes raw device pointers and the current
CUDA stream, and turns status codes into exceptions.  There is no CPU path:
if libdipole.so is missing or cannot be loaded, importing the functions raises.

Method: Barnes-Hut fast summation of regularized dipole sums, forward and
adjoint (Chen, Miller, Gkioulekas, arXiv 2405.16788, Sec. 6 and Alg. 1).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# DIPOLE_LIBRARY selects another build of the library (the checked build,
# libdipole_checked.so); by default the one next to this file.
LIB_PATH = os.environ.get("DIPOLE_LIBRARY") or os.path.join(_HERE, "libdipole.so")

DIPOLE_OK = 0
DIPOLE_EINVAL = -1
DIPOLE_ENOMEM = -2
DIPOLE_ECUDA = -3
DIPOLE_ENONFINITE = -4
DIPOLE_ETRAVERSAL = -5
DIPOLE_ESTATE = -6
DIPOLE_EBOUNDS = -7
DIPOLE_F32 = 0
DIPOLE_BF16 = 1
DIPOLE_BF16_MOMENTS = 2

EXPORTED = ["dipole_build_tree", "dipole_refit", "dipole_forward", "dipole_adjoint",
            "dipole_query_counts", "dipole_sync_status", "dipole_tree_info_get",
            "dipole_tree_export", "dipole_tree_destroy", "dipole_last_error",
            "dipole_kernel_launches", "dipole_forward_noalloc", "dipole_probe_l2",
            "dipole_tree_import", "dipole_forward_planned", "dipole_adjoint_planned",
            "dipole_forward_grad", "dipole_adjoint_grad", "dipole_adjoint_geom",
            "dipole_forward_grid", "dipole_adjoint_acc_size", "dipole_adjoint_stage1",
            "dipole_adjoint_stage2", "dipole_adjoint_queries", "dipole_query_packet_counts",
            "dipole_device_allocations", "dipole_traversal_timer", "dipole_traversal_elapsed",
            "dipole_refit_appearance", "dipole_checked_build", "dipole_set_treelet"]


class DipoleError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


DIPOLE_KERNEL_REGULARIZED = 0
DIPOLE_KERNEL_DESINGULARIZED = 1
_KERNELS = {"regularized": DIPOLE_KERNEL_REGULARIZED, "desingularized": DIPOLE_KERNEL_DESINGULARIZED}


def _kernel_code(kernel) -> int:
    return _KERNELS[kernel] if isinstance(kernel, str) else int(kernel)


class _BuildParams(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int32), ("max_depth", ctypes.c_int32),
                ("kernel", ctypes.c_int32)]


class _TreeInfo(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_nodes", ctypes.c_int64),
                ("channels", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("leaf_size", ctypes.c_int32), ("max_depth", ctypes.c_int32),
                ("bbox_lo", ctypes.c_float * 3), ("bbox_ext", ctypes.c_float),
                ("kernel", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libdipole.so (built by __graft_entry__.build()); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"libdipole.so not found at {path}: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        P, I32, I64, F = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        sig = {
            "dipole_build_tree": [P, P, P, P, I64, P, P, P],
            "dipole_refit": [P, P, I32, I32, P],
            "dipole_forward": [P, P, I64, F, P, P],
            "dipole_forward_noalloc": [P, P, I64, F, P, P],
            "dipole_forward_planned": [P, P, I64, F, P, P, P, P],
            "dipole_adjoint_planned": [P, P, I64, F, P, P, I32, P, P, P],
            "dipole_adjoint": [P, P, I64, F, P, P, I32, P],
            "dipole_query_counts": [P, P, I64, F, P, P],
            "dipole_forward_grad": [P, P, I64, F, P, P, P, P, P],
            "dipole_adjoint_grad": [P, P, I64, F, P, P, P, I32, P, P, P],
            "dipole_adjoint_geom": [P, P, I64, F, P, P, P, P, P, I32, P, P, P],
            "dipole_forward_grid": [P, P, F, P, F, P, P],
            "dipole_sync_status": [P, P],
            "dipole_tree_info_get": [P, P],
            "dipole_tree_export": [P] * 15,
            "dipole_probe_l2": [P, I64, I32, P, P],
            "dipole_tree_import": [P, P, P, P, I64, P, P, P, P, P, P, P, I64, P, P, P],
            "dipole_adjoint_acc_size": [P, P],
            "dipole_adjoint_stage1": [P, P, I64, F, P, P, I32, P, P, P],
            "dipole_adjoint_stage2": [P, P, P, I32, P],
            "dipole_adjoint_queries": [P, P, I64, F, P, P, I32, P],
            "dipole_query_packet_counts": [P, P, I64, F, P, P, P],
            "dipole_traversal_timer": [I32],
            "dipole_refit_appearance": [P, P, I32, I32, I32, P],
            "dipole_traversal_elapsed": [I32, P, P],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.dipole_tree_destroy.argtypes = [P]
        lib.dipole_tree_destroy.restype = None
        lib.dipole_last_error.argtypes = []
        lib.dipole_last_error.restype = ctypes.c_char_p
        lib.dipole_kernel_launches.argtypes = []
        lib.dipole_kernel_launches.restype = ctypes.c_uint64
        lib.dipole_device_allocations.argtypes = []
        lib.dipole_device_allocations.restype = ctypes.c_uint64
        lib.dipole_checked_build.argtypes = []
        lib.dipole_checked_build.restype = ctypes.c_int
        lib.dipole_set_treelet.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        _lib = lib
        return lib


def dipole_last_error() -> str:
    return load_library().dipole_last_error().decode()


def dipole_kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load_library().dipole_kernel_launches())


def dipole_device_allocations() -> int:
    """Device allocations made by the library so far in this process."""
    return int(load_library().dipole_device_allocations())


def dipole_set_treelet(tree: int, enable: bool):
    """Stage the upper tree in shared memory for the value forward (see the header)."""
    _check(load_library().dipole_set_treelet(ctypes.c_void_p(tree), 1 if enable else 0))


def dipole_checked_build() -> bool:
    """True when the loaded library is the checked build (DIPOLE_CHECKED)."""
    return bool(load_library().dipole_checked_build())


TIMER_MODES = {"forward": 0, "adjoint": 1, "counts": 2, "forward_grad": 3, "adjoint_grad": 4,
               "adjoint_geom": 5, "query_grad": 6}


def dipole_traversal_timer(enable: bool):
    """Record CUDA events around every traversal kernel launch (or stop)."""
    _check(load_library().dipole_traversal_timer(int(bool(enable))))


def dipole_traversal_elapsed(mode: str):
    """(total ms, launches) of the traversal kernels of `mode` recorded since
    the last call; waits for them."""
    ms = ctypes.c_float(0.0)
    n = ctypes.c_int64(0)
    _check(load_library().dipole_traversal_elapsed(TIMER_MODES[mode], ctypes.byref(ms),
                                                   ctypes.byref(n)))
    return float(ms.value), int(n.value)


def _check(rc: int):
    if rc != DIPOLE_OK:
        raise DipoleError(rc, dipole_last_error())


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, name: str, dtype=torch.float32, shape=None) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- C names

def dipole_build_tree(points, normals, areas, radii=None, leaf_size=8, max_depth=10,
                      stream=None, kernel="regularized") -> int:
    """Build the octree and node geometry; returns the opaque tree handle.
    kernel: "regularized" (the paper's) or "desingularized" (its ablation)."""
    lib = load_library()
    n = int(points.shape[0])
    pp = _dev(points, "points", shape=(n, 3))
    pn = _dev(normals, "normals", shape=(n, 3))
    pa = _dev(areas, "areas", shape=(n,))
    pr = None if radii is None else _dev(radii, "radii", shape=(n,))
    params = _BuildParams(int(leaf_size), int(max_depth), _kernel_code(kernel))
    h = ctypes.c_void_p()
    _check(lib.dipole_build_tree(pp, pn, pa, pr, n, ctypes.byref(params), _stream(stream),
                                 ctypes.byref(h)))
    return h.value


def _attr_dtype(attrs: torch.Tensor, bf16_moments: bool) -> int:
    dt = {torch.float32: DIPOLE_F32, torch.bfloat16: DIPOLE_BF16}.get(attrs.dtype)
    if dt is None:
        raise TypeError("attrs must be float32 or bfloat16")
    if bf16_moments:
        if dt != DIPOLE_BF16:
            raise TypeError("bf16_moments needs bfloat16 attrs")
        dt = DIPOLE_BF16_MOMENTS
    return dt


def dipole_refit(tree: int, attrs: torch.Tensor, stream=None, bf16_moments: bool = False):
    """Tree update; bf16_moments (bfloat16 attrs only): the value forward reads
    a bf16 copy of the node moments (DIPOLE_BF16_MOMENTS)."""
    if attrs.dim() == 1:
        attrs = attrs[:, None]
    dt = _attr_dtype(attrs, bf16_moments)
    p = _dev(attrs, "attrs", dtype=None)
    _check(load_library().dipole_refit(ctypes.c_void_p(tree), p, int(attrs.shape[1]), dt,
                                       _stream(stream)))


def dipole_refit_appearance(tree: int, attrs: torch.Tensor, geometry_channels: int, stream=None,
                            bf16_moments: bool = False):
    """Refit with channels [geometry_channels, C) interpolated without the
    foreshortening term (the paper's appearance attributes)."""
    if attrs.dim() == 1:
        attrs = attrs[:, None]
    dt = _attr_dtype(attrs, bf16_moments)
    p = _dev(attrs, "attrs", dtype=None)
    _check(load_library().dipole_refit_appearance(ctypes.c_void_p(tree), p, int(attrs.shape[1]),
                                                  dt, int(geometry_channels), _stream(stream)))


def dipole_forward(tree: int, queries: torch.Tensor, beta: float, out: torch.Tensor,
                   stream=None):
    q = int(queries.shape[0])
    _check(load_library().dipole_forward(ctypes.c_void_p(tree), _dev(queries, "queries", shape=(q, 3)),
                                         q, float(beta), _dev(out, "out"), _stream(stream)))


def dipole_forward_noalloc(tree: int, queries: torch.Tensor, beta: float, out: torch.Tensor,
                           stream=None):
    """dipole_forward with its scratch in a static device array: allocates
    nothing, q <= 262144, overlapping calls race (see include/dipole.h)."""
    q = int(queries.shape[0])
    _check(load_library().dipole_forward_noalloc(ctypes.c_void_p(tree),
                                                 _dev(queries, "queries", shape=(q, 3)), q,
                                                 float(beta), _dev(out, "out"), _stream(stream)))


def dipole_adjoint(tree: int, queries: torch.Tensor, beta: float, grad_out: torch.Tensor,
                   grad_attrs: torch.Tensor, accumulate: bool = False, stream=None):
    q = int(queries.shape[0])
    _check(load_library().dipole_adjoint(ctypes.c_void_p(tree), _dev(queries, "queries", shape=(q, 3)),
                                         q, float(beta), _dev(grad_out, "grad_out"),
                                         _dev(grad_attrs, "grad_attrs"), int(bool(accumulate)),
                                         _stream(stream)))


def dipole_adjoint_acc_size(tree: int) -> int:
    """Entries of a stage-1 accumulator for the tree's current channel count."""
    n = ctypes.c_int64(0)
    _check(load_library().dipole_adjoint_acc_size(ctypes.c_void_p(tree), ctypes.byref(n)))
    return int(n.value)


def dipole_adjoint_stage1(tree: int, queries: torch.Tensor, beta: float, grad_out: torch.Tensor,
                          acc: torch.Tensor, accumulate: bool = False, plan=None, stream=None):
    """Stage 1 of the adjoint (node and opened-leaf sums) into acc [acc_size] float."""
    q = int(queries.shape[0])
    pp, pc = _plan_ptrs(plan, q)
    _check(load_library().dipole_adjoint_stage1(
        ctypes.c_void_p(tree), _dev(queries, "queries", shape=(q, 3)), q, float(beta),
        _dev(grad_out, "grad_out"), _dev(acc, "acc", shape=(dipole_adjoint_acc_size(tree),)),
        int(bool(accumulate)), pp, pc, _stream(stream)))


def dipole_adjoint_stage2(tree: int, acc: torch.Tensor, grad_attrs: torch.Tensor,
                          accumulate: bool = False, stream=None):
    """Stage 2 of the adjoint from a (possibly all-reduced) accumulator."""
    _check(load_library().dipole_adjoint_stage2(
        ctypes.c_void_p(tree), _dev(acc, "acc", shape=(dipole_adjoint_acc_size(tree),)),
        _dev(grad_attrs, "grad_attrs"), int(bool(accumulate)), _stream(stream)))


def dipole_adjoint_queries(tree: int, queries: torch.Tensor, beta: float, grad_out: torch.Tensor,
                           grad_queries: torch.Tensor, accumulate: bool = False, stream=None):
    """grad_queries [q, 3] (+)= sum_c grad_out[:, c] grad_x D^c at the queries."""
    q = int(queries.shape[0])
    _check(load_library().dipole_adjoint_queries(
        ctypes.c_void_p(tree), _dev(queries, "queries", shape=(q, 3)), q, float(beta),
        _dev(grad_out, "grad_out"), _dev(grad_queries, "grad_queries", shape=(q, 3)),
        int(bool(accumulate)), _stream(stream)))


class QueryPlan:
    """Caller-owned query plan: the Morton order of a query batch and a record
    of each 32-query packet's walk (its steps and the nodes where it passed
    every 128th step), written by the forward (dipole_forward_planned,
    dipole_forward_grad) and read by the adjoint on the same queries."""

    WORDS_PER_PACKET = 8

    def __init__(self, q: int, device):
        self.q = int(q)
        npk = max((self.q + 31) // 32, 1)
        self.perm = torch.empty(max(self.q, 1), dtype=torch.int32, device=device)
        self.cost = torch.empty(npk * self.WORDS_PER_PACKET, dtype=torch.int32, device=device)


def dipole_forward_planned(tree: int, queries: torch.Tensor, beta: float, out: torch.Tensor,
                           plan: QueryPlan, stream=None):
    q = int(queries.shape[0])
    if plan.q != q:
        raise ValueError("plan was made for another query count")
    _check(load_library().dipole_forward_planned(
        ctypes.c_void_p(tree), _dev(queries, "queries", shape=(q, 3)), q, float(beta),
        _dev(out, "out"), ctypes.c_void_p(plan.perm.data_ptr()),
        ctypes.c_void_p(plan.cost.data_ptr()), _stream(stream)))


def dipole_adjoint_planned(tree: int, queries: torch.Tensor, beta: float, grad_out: torch.Tensor,
                           grad_attrs: torch.Tensor, plan: QueryPlan, accumulate: bool = False,
                           stream=None):
    q = int(queries.shape[0])
    if plan.q != q:
        raise ValueError("plan was made for another query count")
    _check(load_library().dipole_adjoint_planned(
        ctypes.c_void_p(tree), _dev(queries, "queries", shape=(q, 3)), q, float(beta),
        _dev(grad_out, "grad_out"), _dev(grad_attrs, "grad_attrs"), int(bool(accumulate)),
        ctypes.c_void_p(plan.perm.data_ptr()), ctypes.c_void_p(plan.cost.data_ptr()),
        _stream(stream)))


def _opt(t, name, shape=None) -> ctypes.c_void_p:
    return ctypes.c_void_p(None) if t is None else _dev(t, name, shape=shape)


def _plan_ptrs(plan, q):
    if plan is None:
        return ctypes.c_void_p(None), ctypes.c_void_p(None)
    if plan.q != q:
        raise ValueError("plan was made for another query count")
    return ctypes.c_void_p(plan.perm.data_ptr()), ctypes.c_void_p(plan.cost.data_ptr())


def dipole_forward_grad(tree: int, queries: torch.Tensor, beta: float, out, grad_x: torch.Tensor,
                        plan: QueryPlan | None = None, stream=None):
    """D (into `out`, may be None) and its query-position gradient into
    grad_x [q, C, 3]; with `plan`, also record the query plan."""
    q = int(queries.shape[0])
    pp, pc = _plan_ptrs(plan, q)
    _check(load_library().dipole_forward_grad(
        ctypes.c_void_p(tree), _dev(queries, "queries", shape=(q, 3)), q, float(beta),
        _opt(out, "out"), _dev(grad_x, "grad_x"), pp, pc, _stream(stream)))


def dipole_adjoint_grad(tree: int, queries: torch.Tensor, beta: float, grad_out, grad_grad,
                        grad_attrs: torch.Tensor, accumulate: bool = False,
                        plan: QueryPlan | None = None, stream=None):
    """dL/dmu for dL/dD = grad_out [q, C] and dL/d(grad D) = grad_grad [q, C, 3]
    (either may be None); with `plan` from dipole_forward_grad on these queries."""
    q = int(queries.shape[0])
    pp, pc = _plan_ptrs(plan, q)
    _check(load_library().dipole_adjoint_grad(
        ctypes.c_void_p(tree), _dev(queries, "queries", shape=(q, 3)), q, float(beta),
        _opt(grad_out, "grad_out"), _opt(grad_grad, "grad_grad"), _dev(grad_attrs, "grad_attrs"),
        int(bool(accumulate)), pp, pc, _stream(stream)))


def dipole_adjoint_geom(tree: int, queries: torch.Tensor, beta: float, grad_out, grad_grad,
                        grad_attrs, grad_normals, grad_radii, accumulate: bool = False,
                        plan: QueryPlan | None = None, stream=None):
    """dL/dmu [n, C], dL/dn [n, 3], dL/deps [n] (each may be None) for upstream
    gradients of D and grad D (either may be None)."""
    q = int(queries.shape[0])
    pp, pc = _plan_ptrs(plan, q)
    _check(load_library().dipole_adjoint_geom(
        ctypes.c_void_p(tree), _dev(queries, "queries", shape=(q, 3)), q, float(beta),
        _opt(grad_out, "grad_out"), _opt(grad_grad, "grad_grad"), _opt(grad_attrs, "grad_attrs"),
        _opt(grad_normals, "grad_normals"), _opt(grad_radii, "grad_radii"),
        int(bool(accumulate)), pp, pc, _stream(stream)))


def dipole_forward_grid(tree: int, lo, spacing: float, dims, beta: float, out: torch.Tensor,
                        stream=None):
    """D on the grid lo + spacing * (i, j, k): out [dims[2], dims[1], dims[0], C]."""
    lo_h = np.ascontiguousarray(np.asarray(lo, np.float32).reshape(3))
    dims_h = np.ascontiguousarray(np.asarray(dims, np.int64).reshape(3))
    _check(load_library().dipole_forward_grid(
        ctypes.c_void_p(tree), lo_h.ctypes.data_as(ctypes.c_void_p), float(spacing),
        dims_h.ctypes.data_as(ctypes.c_void_p), float(beta), _dev(out, "out"), _stream(stream)))


def dipole_query_counts(tree: int, queries: torch.Tensor, beta: float, counts: torch.Tensor,
                        stream=None):
    q = int(queries.shape[0])
    _check(load_library().dipole_query_counts(ctypes.c_void_p(tree),
                                              _dev(queries, "queries", shape=(q, 3)), q,
                                              float(beta),
                                              _dev(counts, "counts", dtype=torch.int32,
                                                   shape=(q, 3)),
                                              _stream(stream)))


def dipole_query_packet_counts(tree: int, queries: torch.Tensor, beta: float,
                               packet_counts: torch.Tensor, counts=None, stream=None):
    """Per 32-query packet {warp steps, far steps, opened-leaf points, lanes}."""
    q = int(queries.shape[0])
    _check(load_library().dipole_query_packet_counts(
        ctypes.c_void_p(tree), _dev(queries, "queries", shape=(q, 3)), q, float(beta),
        ctypes.c_void_p(None) if counts is None else _dev(counts, "counts", dtype=torch.int32,
                                                          shape=(q, 3)),
        _dev(packet_counts, "packet_counts", dtype=torch.int32, shape=((q + 31) // 32, 4)),
        _stream(stream)))


def dipole_sync_status(tree: int, stream=None):
    _check(load_library().dipole_sync_status(ctypes.c_void_p(tree), _stream(stream)))


def dipole_tree_info_get(tree: int) -> dict:
    info = _TreeInfo()
    _check(load_library().dipole_tree_info_get(ctypes.c_void_p(tree), ctypes.byref(info)))
    return dict(n_points=info.n_points, n_nodes=info.n_nodes, channels=info.channels,
                dtype=info.dtype, leaf_size=info.leaf_size, max_depth=info.max_depth,
                bbox_lo=list(info.bbox_lo), bbox_ext=info.bbox_ext, kernel=info.kernel)


def dipole_tree_export(tree: int, moments: bool = False, stream=None) -> dict:
    info = dipole_tree_info_get(tree)
    n, nn, C = info["n_points"], info["n_nodes"], info["channels"]
    o = dict(code=np.zeros(n, np.uint32), perm=np.zeros(n, np.uint32),
             first=np.zeros(nn, np.int32), count=np.zeros(nn, np.int32),
             level=np.zeros(nn, np.int32), parent=np.zeros(nn, np.int32),
             skip=np.zeros(nn, np.int32), is_leaf=np.zeros(nn, np.int32),
             cen32=np.zeros((nn, 3), np.float32), r32=np.zeros(nn, np.float32),
             area=np.zeros(nn, np.float64), eps=np.zeros(nn, np.float32))
    if moments:
        o["moments"] = np.zeros((nn, 3 * C), np.float32)
    keys = ["code", "perm", "first", "count", "level", "parent", "skip", "is_leaf", "cen32",
            "r32", "area", "eps", "moments"]
    ptrs = [o[k].ctypes.data_as(ctypes.c_void_p) if k in o else None for k in keys]
    _check(load_library().dipole_tree_export(ctypes.c_void_p(tree), *ptrs, _stream(stream)))
    return o


def dipole_probe_l2(buf: torch.Tensor, passes: int, sink: torch.Tensor, stream=None):
    """Diagnostics: read `buf` `passes` times with L2-only loads (for timing)."""
    _check(load_library().dipole_probe_l2(ctypes.c_void_p(buf.data_ptr()),
                                          buf.numel() * buf.element_size(), int(passes),
                                          ctypes.c_void_p(sink.data_ptr()), _stream(stream)))


def dipole_tree_import(points, normals, areas, radii, exported: dict, leaf_size=8, max_depth=10,
                       stream=None, kernel="regularized") -> int:
    """Rebuild a tree from dipole_tree_export's arrays (host numpy) and the
    point inputs (CUDA tensors); returns the tree handle."""
    lib = load_library()
    n = int(points.shape[0])
    host = {k: np.ascontiguousarray(exported[k], dtype=np.int32)
            for k in ("first", "count", "level", "skip", "is_leaf")}
    perm = np.ascontiguousarray(exported["perm"], dtype=np.uint32)
    code = exported.get("code")
    code = None if code is None else np.ascontiguousarray(code, dtype=np.uint32)
    nn = int(host["first"].shape[0])
    hp = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    params = _BuildParams(int(leaf_size), int(max_depth), _kernel_code(kernel))
    h = ctypes.c_void_p()
    _check(lib.dipole_tree_import(_dev(points, "points", shape=(n, 3)),
                                  _dev(normals, "normals", shape=(n, 3)),
                                  _dev(areas, "areas", shape=(n,)),
                                  None if radii is None else _dev(radii, "radii", shape=(n,)), n,
                                  hp(code), hp(perm), hp(host["first"]), hp(host["count"]),
                                  hp(host["level"]), hp(host["skip"]), hp(host["is_leaf"]), nn,
                                  ctypes.byref(params), _stream(stream), ctypes.byref(h)))
    return h.value


def dipole_tree_destroy(tree: int):
    if tree:
        load_library().dipole_tree_destroy(ctypes.c_void_p(tree))


# ---------------------------------------------------------------- objects

class DipoleTree:
    """Owns a dipole_tree handle.  Inputs are float32 CUDA tensors in the
    caller's point order; outputs come back in that order."""

    def __init__(self, points, normals, areas, radii=None, leaf_size=8, max_depth=10,
                 stream=None, kernel="regularized"):
        self.n = int(points.shape[0])
        # kernels still read the inputs after the build call returns (stream order)
        self._inputs = (points, normals, areas, radii)
        self.handle = dipole_build_tree(points, normals, areas, radii, leaf_size, max_depth,
                                        stream, kernel)
        self.C = 0
        self.device = points.device

    @classmethod
    def from_export(cls, points, normals, areas, radii, exported: dict, leaf_size=8, max_depth=10,
                    stream=None, kernel="regularized") -> "DipoleTree":
        """A tree rebuilt from dipole_tree_export's arrays (checkpoint / resume)."""
        self = cls.__new__(cls)
        self.n = int(points.shape[0])
        self._inputs = (points, normals, areas, radii)
        self.handle = dipole_tree_import(points, normals, areas, radii, exported, leaf_size,
                                         max_depth, stream, kernel)
        self.C = 0
        self.device = points.device
        return self

    def close(self):
        if getattr(self, "handle", None):
            dipole_tree_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self) -> dict:
        return dipole_tree_info_get(self.handle)

    def refit(self, attrs: torch.Tensor, stream=None, geometry_channels: int | None = None,
              bf16_moments: bool = False):
        """Tree update (eq. farfield_dipole_features).  geometry_channels = G < C:
        channels [G, C) skip the foreshortening term (appearance attributes).
        bf16_moments (bfloat16 attrs): the value forward reads bf16 node moments."""
        if attrs.dim() == 1:
            attrs = attrs[:, None]
        if attrs.shape[0] != self.n:
            raise ValueError("attrs must have one row per point")
        attrs = attrs.contiguous()
        if geometry_channels is None:
            dipole_refit(self.handle, attrs, stream, bf16_moments)
        else:
            dipole_refit_appearance(self.handle, attrs, geometry_channels, stream, bf16_moments)
        self.C = int(attrs.shape[1])
        self._attrs = attrs

    def forward(self, queries: torch.Tensor, beta: float, out: torch.Tensor | None = None,
                plan: QueryPlan | None = None, stream=None) -> torch.Tensor:
        """Primal queries; with `plan`, also record the query plan for the adjoint."""
        if self.C == 0:
            raise DipoleError(DIPOLE_ESTATE, "refit first")
        if out is None:
            out = torch.empty((queries.shape[0], self.C), device=queries.device,
                              dtype=torch.float32)
        if plan is None:
            dipole_forward(self.handle, queries, beta, out, stream)
        else:
            dipole_forward_planned(self.handle, queries, beta, out, plan, stream)
        return out

    def adjoint(self, queries: torch.Tensor, beta: float, grad_out: torch.Tensor,
                grad_attrs: torch.Tensor | None = None, accumulate: bool = False,
                plan: QueryPlan | None = None, stream=None) -> torch.Tensor:
        """Two-stage adjoint; with `plan` from a forward on the same queries,
        reuse its query order and schedule the longest packets first."""
        if self.C == 0:
            raise DipoleError(DIPOLE_ESTATE, "refit first")
        if grad_attrs is None:
            grad_attrs = torch.empty((self.n, self.C), device=queries.device, dtype=torch.float32)
            accumulate = False
        if plan is None:
            dipole_adjoint(self.handle, queries, beta, grad_out.contiguous(), grad_attrs,
                           accumulate, stream)
        else:
            dipole_adjoint_planned(self.handle, queries, beta, grad_out.contiguous(), grad_attrs,
                                   plan, accumulate, stream)
        return grad_attrs

    def forward_grad(self, queries: torch.Tensor, beta: float, value: bool = True,
                     plan: QueryPlan | None = None, stream=None):
        """(D [q, C] or None, grad_x D [q, C, 3]) at the queries."""
        if self.C == 0:
            raise DipoleError(DIPOLE_ESTATE, "refit first")
        q = queries.shape[0]
        out = torch.empty((q, self.C), device=queries.device, dtype=torch.float32) if value else None
        gx = torch.empty((q, self.C, 3), device=queries.device, dtype=torch.float32)
        dipole_forward_grad(self.handle, queries, beta, out, gx, plan, stream)
        return out, gx

    def adjoint_grad(self, queries: torch.Tensor, beta: float, grad_out=None, grad_grad=None,
                     grad_attrs: torch.Tensor | None = None, accumulate: bool = False,
                     plan: QueryPlan | None = None, stream=None) -> torch.Tensor:
        """dL/dmu for upstream gradients of D and of grad_x D (either may be None)."""
        if self.C == 0:
            raise DipoleError(DIPOLE_ESTATE, "refit first")
        if grad_attrs is None:
            grad_attrs = torch.empty((self.n, self.C), device=queries.device, dtype=torch.float32)
            accumulate = False
        c = lambda t: None if t is None else t.to(torch.float32).contiguous()
        dipole_adjoint_grad(self.handle, queries, beta, c(grad_out), c(grad_grad), grad_attrs,
                            accumulate, plan, stream)
        return grad_attrs

    def adjoint_geom(self, queries: torch.Tensor, beta: float, grad_out=None, grad_grad=None,
                     attrs: bool = True, normals: bool = True, radii: bool = True,
                     plan: QueryPlan | None = None, stream=None):
        """(dL/dmu [n, C], dL/dn [n, 3], dL/deps [n]) for upstream gradients of D
        and of grad_x D; an output not asked for is None."""
        if self.C == 0:
            raise DipoleError(DIPOLE_ESTATE, "refit first")
        dev = queries.device
        gm = torch.empty((self.n, self.C), device=dev, dtype=torch.float32) if attrs else None
        gn = torch.empty((self.n, 3), device=dev, dtype=torch.float32) if normals else None
        ge = torch.empty((self.n,), device=dev, dtype=torch.float32) if radii else None
        c = lambda t: None if t is None else t.to(torch.float32).contiguous()
        dipole_adjoint_geom(self.handle, queries, beta, c(grad_out), c(grad_grad), gm, gn, ge,
                            False, plan, stream)
        return gm, gn, ge

    def forward_grid(self, lo, spacing: float, dims, beta: float, stream=None) -> torch.Tensor:
        """D on a dense grid: [dims[2], dims[1], dims[0], C] (x fastest)."""
        if self.C == 0:
            raise DipoleError(DIPOLE_ESTATE, "refit first")
        nx, ny, nz = (int(d) for d in dims)
        out = torch.empty((nz, ny, nx, self.C), device=self.device, dtype=torch.float32)
        dipole_forward_grid(self.handle, lo, spacing, (nx, ny, nz), beta, out, stream)
        return out

    def adjoint_queries(self, queries: torch.Tensor, beta: float, grad_out: torch.Tensor,
                        stream=None) -> torch.Tensor:
        """dL/dx [q, 3] = sum_c grad_out[:, c] grad_x D^c (the library does the sum)."""
        if self.C == 0:
            raise DipoleError(DIPOLE_ESTATE, "refit first")
        gq = torch.empty((queries.shape[0], 3), device=queries.device, dtype=torch.float32)
        dipole_adjoint_queries(self.handle, queries, beta, grad_out.to(torch.float32).contiguous(),
                               gq, False, stream)
        return gq

    def adjoint_acc_size(self) -> int:
        return dipole_adjoint_acc_size(self.handle)

    def adjoint_stage1(self, queries: torch.Tensor, beta: float, grad_out: torch.Tensor,
                       acc: torch.Tensor | None = None, accumulate: bool = False,
                       plan: QueryPlan | None = None, stream=None) -> torch.Tensor:
        """Stage 1 of the adjoint into an accumulator (summable across ranks)."""
        if self.C == 0:
            raise DipoleError(DIPOLE_ESTATE, "refit first")
        if acc is None:
            acc = torch.empty(self.adjoint_acc_size(), device=queries.device, dtype=torch.float32)
            accumulate = False
        dipole_adjoint_stage1(self.handle, queries, beta, grad_out.to(torch.float32).contiguous(),
                              acc, accumulate, plan, stream)
        return acc

    def adjoint_stage2(self, acc: torch.Tensor, grad_attrs: torch.Tensor | None = None,
                       accumulate: bool = False, stream=None) -> torch.Tensor:
        if grad_attrs is None:
            grad_attrs = torch.empty((self.n, self.C), device=acc.device, dtype=torch.float32)
            accumulate = False
        dipole_adjoint_stage2(self.handle, acc, grad_attrs, accumulate, stream)
        return grad_attrs

    def query_counts(self, queries: torch.Tensor, beta: float, stream=None) -> torch.Tensor:
        counts = torch.empty((queries.shape[0], 3), device=queries.device, dtype=torch.int32)
        dipole_query_counts(self.handle, queries, beta, counts, stream)
        return counts

    def sync_status(self, stream=None):
        dipole_sync_status(self.handle, stream)

    def export(self, moments: bool = False) -> dict:
        return dipole_tree_export(self.handle, moments)


class DipoleSum(torch.autograd.Function):
    """D = dipole sum of `attrs` at `queries` (Barnes-Hut, Alg. 1).  Forward runs
    the tree update then the primal queries; backward runs the two-stage adjoint
    (Sec. 6.2), recomputing the traversal instead of storing interaction lists."""

    @staticmethod
    def forward(ctx, attrs, tree: DipoleTree, queries, beta: float):
        tree.refit(attrs)
        plan = QueryPlan(queries.shape[0], queries.device)
        out = tree.forward(queries, beta, plan=plan)
        ctx.plan = plan
        ctx.tree = tree
        ctx.beta = float(beta)
        ctx.C = tree.C
        ctx.attr_dtype = attrs.dtype
        ctx.attr_shape = attrs.shape
        ctx.save_for_backward(queries)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (queries,) = ctx.saved_tensors
        tree = ctx.tree
        if tree.C != ctx.C:
            raise DipoleError(DIPOLE_ESTATE, "the tree was refit with another channel count "
                                             "between forward and backward")
        go = grad_out.to(torch.float32).contiguous()
        g = gq = None
        if ctx.needs_input_grad[0]:
            g = tree.adjoint(queries, ctx.beta, go, plan=ctx.plan)
            g = g.to(ctx.attr_dtype).reshape(ctx.attr_shape)
        if ctx.needs_input_grad[2]:
            # dL/dx_j = sum_c dL/dD^c grad_x D^c(x_j), summed in the library; the
            # tree still holds the forward's moments (refit in forward, not since)
            gq = tree.adjoint_queries(queries.detach(), ctx.beta, go).to(queries.dtype)
        return g, None, gq, None


class DipoleSumGrad(torch.autograd.Function):
    """(D, grad_x D) of `attrs` at `queries`: the dipole sum and its spatial
    gradient as functions of the attributes (both linear in them).  Backward
    is the two-stage adjoint of both outputs; queries get no gradient."""

    @staticmethod
    def forward(ctx, attrs, tree: DipoleTree, queries, beta: float, refit: bool = True):
        if refit:
            tree.refit(attrs)
        elif tree.C != attrs.reshape(attrs.shape[0], -1).shape[1]:
            raise DipoleError(DIPOLE_ESTATE, "refit=False needs the tree refit with these attrs")
        plan = QueryPlan(queries.shape[0], queries.device)
        out, gx = tree.forward_grad(queries, beta, value=True, plan=plan)
        ctx.plan = plan
        ctx.tree = tree
        ctx.beta = float(beta)
        ctx.C = tree.C
        ctx.attr_dtype = attrs.dtype
        ctx.attr_shape = attrs.shape
        ctx.save_for_backward(queries)
        return out, gx

    @staticmethod
    def backward(ctx, grad_out, grad_gx):
        (queries,) = ctx.saved_tensors
        tree = ctx.tree
        if tree.C != ctx.C:
            raise DipoleError(DIPOLE_ESTATE, "the tree was refit with another channel count "
                                             "between forward and backward")
        if grad_out is None and grad_gx is None:
            return None, None, None, None, None
        g = tree.adjoint_grad(queries, ctx.beta, grad_out, grad_gx, plan=ctx.plan)
        return g.to(ctx.attr_dtype).reshape(ctx.attr_shape), None, None, None, None


def dipole_sum_and_grad(attrs: torch.Tensor, tree: DipoleTree, queries: torch.Tensor,
                        beta: float = 2.0, refit: bool = True):
    """(D [q, C], grad_x D [q, C, 3]), differentiable in attrs.  refit=False
    skips the tree update when the tree already holds these attrs (a second
    query batch in the same step); the caller guarantees that."""
    return DipoleSumGrad.apply(attrs, tree, queries, beta, refit)


class DipoleField(torch.autograd.Function):
    """The dipole sum (and optionally its spatial gradient) differentiable in
    the point normals, radii and attributes, as trained by the paper's inverse
    rendering (positions and areas are fixed).  Forward builds the tree from
    the current normals and radii, refits the attributes and queries; backward
    is the adjoint of every output with respect to all three (and the queries
    get sum_c dL/dD^c grad D^c when they require a gradient)."""

    @staticmethod
    def forward(ctx, points, normals, areas, radii, attrs, queries, beta: float, with_grad: bool,
                leaf_size: int):
        tree = DipoleTree(points.detach(), normals.detach().contiguous(), areas.detach(),
                          None if radii is None else radii.detach().contiguous(),
                          leaf_size=leaf_size)
        tree.refit(attrs.detach())
        plan = QueryPlan(queries.shape[0], queries.device)
        q = queries.detach().contiguous()
        if with_grad:
            d, gx = tree.forward_grad(q, beta, value=True, plan=plan)
        else:
            d, gx = tree.forward(q, beta, plan=plan), None
        ctx.tree, ctx.plan, ctx.beta, ctx.with_grad = tree, plan, float(beta), with_grad
        ctx.attr_dtype, ctx.attr_shape = attrs.dtype, attrs.shape
        ctx.has_radii = radii is not None
        ctx.save_for_backward(q)
        return (d, gx) if with_grad else d

    @staticmethod
    def backward(ctx, grad_out, grad_gx=None):
        (q,) = ctx.saved_tensors
        tree = ctx.tree
        need = ctx.needs_input_grad
        gn = ge = gm = gq = None
        if need[1] or need[3] or need[4]:
            gm, gn, ge = tree.adjoint_geom(q, ctx.beta, grad_out, grad_gx if ctx.with_grad else None,
                                           attrs=need[4], normals=need[1],
                                           radii=need[3] and ctx.has_radii, plan=ctx.plan)
            if gm is not None:
                gm = gm.to(ctx.attr_dtype).reshape(ctx.attr_shape)
        if need[5]:
            if ctx.with_grad and grad_gx is not None and bool(torch.any(grad_gx != 0)):
                raise NotImplementedError("second derivatives in the query position")
            gq = tree.adjoint_queries(q, ctx.beta, grad_out)
        return None, gn, None, ge, gm, gq, None, None, None


def dipole_field(points, normals, areas, radii, attrs, queries, beta: float = 2.0,
                 with_grad: bool = False, leaf_size: int = 8):
    """D [q, C] (or (D, grad_x D [q, C, 3]) with with_grad), differentiable in
    normals, radii, attrs (and, for D, the queries)."""
    return DipoleField.apply(points, normals, areas, radii, attrs, queries, beta, with_grad,
                             leaf_size)


def dipole_sum(attrs: torch.Tensor, tree: DipoleTree, queries: torch.Tensor, beta: float = 2.0):
    return DipoleSum.apply(attrs, tree, queries, beta)
