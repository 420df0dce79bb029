"""Oracle for the regularized dipole sum: a plain double-precision CPU statement.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the library's product
path never does.  It shares no code with the CUDA library; both sides only take
their inputs from the seeded generators in ``paper_2405_16788_gb300.synthetic``.

Every function cites the part of the paper (arXiv 2405.16788) that it states:
see ``dipole_oracle.c`` for the list of readings taken where the paper is
silent.  Parity is pinned by ``tests/test_oracle_pins.py`` (closed forms, the
Gauss lemma, Prop. 1 and Prop. 2, brute-force limits of Barnes-Hut, the
adjoint identity and tree invariants on exhaustive small cases).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dipole_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: the Morton quantisation, the far test and the node radius
# are specified operation by operation (no fused multiply-add contraction).
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
          "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile dipole_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_F = ctypes.c_float


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_num_threads.restype = _I
        lib.orc_rho.restype = ctypes.c_double
        lib.orc_rho.argtypes = [ctypes.c_double]
        lib.orc_interleave.restype = ctypes.c_uint32
        lib.orc_interleave.argtypes = [ctypes.c_uint32] * 3
        lib.orc_morton.argtypes = [_I64, _P, _P, _P]
        lib.orc_brute_forward.argtypes = [_I64, _P, _P, _P, _P, _I, _P, _I64, _P, _P]
        lib.orc_brute_adjoint.argtypes = [_I64, _P, _P, _P, _P, _I, _I64, _P, _P, _P]
        lib.orc_brute_forward_app.argtypes = [_I64, _P, _P, _P, _P, _I, _I, _P, _I64, _P, _P]
        lib.orc_brute_adjoint_app.argtypes = [_I64, _P, _P, _P, _P, _I, _I, _I64, _P, _P, _P]
        lib.orc_tree_set_geometry_channels.argtypes = [_P, _I]
        lib.orc_bh_near_ties.argtypes = [_P, _I64, _P, _F, _P]
        lib.orc_tree_build.restype = _P
        lib.orc_tree_build.argtypes = [_I64, _P, _P, _P, _P, _I, _I]
        lib.orc_tree_free.argtypes = [_P]
        lib.orc_tree_num_nodes.restype = _I64
        lib.orc_tree_num_nodes.argtypes = [_P]
        lib.orc_tree_export.argtypes = [_P] * 15
        lib.orc_tree_update.argtypes = [_P, _P, _I]
        lib.orc_round_bf16_n.argtypes = [_I64, _P, _P]
        lib.orc_tree_round_moments_bf16.argtypes = [_P]
        lib.orc_bh_forward_bf16.argtypes = [_P, _I64, _P, _F, _P, _P, _P]
        lib.orc_bh_forward.argtypes = [_P, _I64, _P, _F, _P, _P]
        lib.orc_bh_adjoint.argtypes = [_P, _I64, _P, _F, _P, _P]
        lib.orc_brute_forward_grad.argtypes = [_I64, _P, _P, _P, _P, _I, _P, _I64, _P, _P]
        lib.orc_bh_forward_grad.argtypes = [_P, _I64, _P, _F, _P]
        lib.orc_bh_adjoint_grad.argtypes = [_P, _I64, _P, _F, _P, _P, _P]
        lib.orc_brute_adjoint_geom.argtypes = [_I64, _P, _P, _P, _P, _I, _P, _I64, _P, _P, _P,
                                               _P, _P, _P]
        lib.orc_bh_adjoint_geom.argtypes = [_P, _I64, _P, _F, _P, _P, _P, _P, _P]
        lib.orc_set_kernel.argtypes = [_I]
        lib.orc_far_test.restype = _I
        lib.orc_far_test.argtypes = [_P, _P, _F, _F]
        _lib = lib
        return lib


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().orc_num_threads())


def rho(t: float) -> float:
    """rho(t) = erf(t) - 2t/sqrt(pi) exp(-t^2); Sec. 4.1, eq. (regularized_poisson)."""
    return float(_load().orc_rho(float(t)))


def interleave(qx: int, qy: int, qz: int) -> int:
    """30-bit Morton interleave: x bit k -> 3k+2, y -> 3k+1, z -> 3k."""
    return int(_load().orc_interleave(qx, qy, qz))


def morton(points):
    """Bounding cube and codes in input order: returns (lo[3], ext, codes[n])."""
    p = _f32(points)
    n = p.shape[0]
    lo_ext = np.zeros(4, np.float32)
    codes = np.zeros(n, np.uint32)
    _load().orc_morton(n, _ptr(p), _ptr(lo_ext), _ptr(codes))
    return lo_ext[:3].copy(), float(lo_ext[3]), codes


def round_bf16(x):
    """x rounded to float and then to bfloat16, nearest even (reading R13), as float64."""
    x = np.ascontiguousarray(x, np.float64)
    out = np.empty_like(x)
    _load().orc_round_bf16_n(x.size, _ptr(x), _ptr(out))
    return out


def brute_forward(points, normals, areas, eps, mu, queries):
    """Plain O(NQ) sum, eq. (dipole_sum)/(appearance_features): out [Q, C] float64."""
    p, nr, a = _f32(points), _f32(normals), _f32(areas)
    e = None if eps is None else _f32(eps)
    mu = _f32(mu)
    if mu.ndim == 1:
        mu = mu[:, None]
    q = _f32(queries)
    n, C, nq = p.shape[0], mu.shape[1], q.shape[0]
    out = np.zeros((nq, C), np.float64)
    _load().orc_brute_forward(n, _ptr(p), _ptr(nr), _ptr(a), _ptr(e), C, _ptr(mu), nq, _ptr(q),
                              _ptr(out))
    return out


def brute_adjoint(points, normals, areas, eps, queries, g):
    """dL/dmu [N, C] float64 for dL/dD = g [Q, C]: the transpose of brute_forward."""
    p, nr, a = _f32(points), _f32(normals), _f32(areas)
    e = None if eps is None else _f32(eps)
    q = _f32(queries)
    g = _f64(g)
    if g.ndim == 1:
        g = g[:, None]
    n, nq, C = p.shape[0], q.shape[0], g.shape[1]
    out = np.zeros((n, C), np.float64)
    _load().orc_brute_adjoint(n, _ptr(p), _ptr(nr), _ptr(a), _ptr(e), C, nq, _ptr(q), _ptr(g),
                              _ptr(out))
    return out


def brute_forward_app(points, normals, areas, eps, mu, queries, geometry_channels):
    """Plain O(NQ) sum with channels [geometry_channels, C) interpolated without
    the foreshortening term (reading R12 of dipole_oracle.c): out [Q, C] float64."""
    p, nr, a = _f32(points), _f32(normals), _f32(areas)
    e = None if eps is None else _f32(eps)
    mu = _f32(mu)
    if mu.ndim == 1:
        mu = mu[:, None]
    q = _f32(queries)
    n, C, nq = p.shape[0], mu.shape[1], q.shape[0]
    out = np.zeros((nq, C), np.float64)
    _load().orc_brute_forward_app(n, _ptr(p), _ptr(nr), _ptr(a), _ptr(e), C,
                                  int(geometry_channels), _ptr(mu), nq, _ptr(q), _ptr(out))
    return out


def brute_adjoint_app(points, normals, areas, eps, queries, g, geometry_channels):
    """The transpose of brute_forward_app: dL/dmu [N, C] float64."""
    p, nr, a = _f32(points), _f32(normals), _f32(areas)
    e = None if eps is None else _f32(eps)
    q = _f32(queries)
    g = _f64(g)
    if g.ndim == 1:
        g = g[:, None]
    n, nq, C = p.shape[0], q.shape[0], g.shape[1]
    out = np.zeros((n, C), np.float64)
    _load().orc_brute_adjoint_app(n, _ptr(p), _ptr(nr), _ptr(a), _ptr(e), C,
                                  int(geometry_channels), nq, _ptr(q), _ptr(g), _ptr(out))
    return out


def brute_forward_grad(points, normals, areas, eps, mu, queries):
    """Plain O(NQ) spatial gradient of the dipole sum (reading R9 of dipole_oracle.c): [Q, C, 3]."""
    p, nr, a = _f32(points), _f32(normals), _f32(areas)
    e = None if eps is None else _f32(eps)
    mu = _f32(mu)
    if mu.ndim == 1:
        mu = mu[:, None]
    q = _f32(queries)
    n, C, nq = p.shape[0], mu.shape[1], q.shape[0]
    out = np.zeros((nq, C, 3), np.float64)
    _load().orc_brute_forward_grad(n, _ptr(p), _ptr(nr), _ptr(a), _ptr(e), C, _ptr(mu), nq,
                                   _ptr(q), _ptr(out))
    return out


def brute_adjoint_geom(points, normals, areas, eps, mu, queries, g=None, gg=None):
    """Plain O(NQ) gradients of L(D, grad D) with respect to mu, the normals and
    eps (readings R9, R10 of dipole_oracle.c): (dmu [N, C], dn [N, 3], deps [N]) float64."""
    p, nr, a = _f32(points), _f32(normals), _f32(areas)
    e = None if eps is None else _f32(eps)
    mu = _f32(mu)
    if mu.ndim == 1:
        mu = mu[:, None]
    q = _f32(queries)
    n, C, nq = p.shape[0], mu.shape[1], q.shape[0]
    g64 = None if g is None else _f64(np.asarray(g).reshape(nq, C))
    gg64 = None if gg is None else _f64(np.asarray(gg).reshape(nq, C, 3))
    dmu = np.zeros((n, C), np.float64)
    dn = np.zeros((n, 3), np.float64)
    deps = np.zeros(n, np.float64)
    _load().orc_brute_adjoint_geom(n, _ptr(p), _ptr(nr), _ptr(a), _ptr(e), C, _ptr(mu), nq,
                                   _ptr(q), _ptr(g64), _ptr(gg64), _ptr(dmu), _ptr(dn),
                                   _ptr(deps))
    return dmu, dn, deps


class kernel:
    """Context manager selecting the oracle's kernel (reading R11 of dipole_oracle.c):
    "regularized" (the paper's, the default) or "desingularized"."""

    _codes = {"regularized": 0, "desingularized": 1}

    def __init__(self, name: str):
        self.code = self._codes[name]

    def __enter__(self):
        _load().orc_set_kernel(self.code)
        return self

    def __exit__(self, *exc):
        _load().orc_set_kernel(0)
        return False


def far_test(x, c, r, beta) -> bool:
    """The far test of Alg. 1 in the float operation order the oracle uses."""
    xx, cc = _f32(x), _f32(c)
    return bool(_load().orc_far_test(_ptr(xx), _ptr(cc), float(r), float(beta)))


class Tree:
    """CPU octree, node aggregates and Barnes-Hut queries (Sec. 6, Alg. 1)."""

    def __init__(self, points, normals, areas, eps=None, leaf_size=8, max_depth=10):
        lib = _load()
        self._p, self._n, self._a = _f32(points), _f32(normals), _f32(areas)
        self._e = None if eps is None else _f32(eps)
        self.n = self._p.shape[0]
        h = lib.orc_tree_build(self.n, _ptr(self._p), _ptr(self._n), _ptr(self._a),
                               _ptr(self._e), int(leaf_size), int(max_depth))
        if not h:
            raise ValueError("oracle tree build rejected its arguments")
        self._h = ctypes.c_void_p(h)
        self.nn = int(lib.orc_tree_num_nodes(self._h))
        self.C = None

    def close(self):
        if getattr(self, "_h", None):
            _load().orc_tree_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def export(self) -> dict:
        """All integer arrays and node geometry as numpy arrays."""
        n, nn = self.n, self.nn
        o = dict(lo_ext=np.zeros(4, np.float32), code=np.zeros(n, np.uint32),
                 perm=np.zeros(n, np.uint32), first=np.zeros(nn, np.int32),
                 count=np.zeros(nn, np.int32), level=np.zeros(nn, np.int32),
                 parent=np.zeros(nn, np.int32), skip=np.zeros(nn, np.int32),
                 is_leaf=np.zeros(nn, np.int32), area=np.zeros(nn, np.float64),
                 cen=np.zeros((nn, 3), np.float64), eps=np.zeros(nn, np.float64),
                 cen32=np.zeros((nn, 3), np.float32), r32=np.zeros(nn, np.float32))
        keys = ["lo_ext", "code", "perm", "first", "count", "level", "parent", "skip",
                "is_leaf", "area", "cen", "eps", "cen32", "r32"]
        _load().orc_tree_export(self._h, *[_ptr(o[k]) for k in keys])
        return o

    def update(self, mu, geometry_channels=None, bf16_moments=False):
        """Tree update of the node moments, eq. (farfield_dipole_features).  With
        geometry_channels = G < C, channels [G, C) are interpolated without the
        foreshortening term (reading R12).  bf16_moments: the far field of
        forward() uses the node sums rounded to float, then to bf16 (reading R13)."""
        mu = _f32(mu)
        if mu.ndim == 1:
            mu = mu[:, None]
        if mu.shape[0] != self.n:
            raise ValueError("mu must have one row per point")
        self.C = mu.shape[1]
        _load().orc_tree_update(self._h, _ptr(mu), self.C)
        self.G = self.C if geometry_channels is None else int(geometry_channels)
        if not 0 <= self.G <= self.C:
            raise ValueError("geometry_channels must be in [0, C]")
        _load().orc_tree_set_geometry_channels(self._h, self.G)
        self.bf16_moments = bool(bf16_moments)
        if bf16_moments:
            _load().orc_tree_round_moments_bf16(self._h)

    def _dipole_only(self):
        if getattr(self, "G", self.C) != self.C:
            raise NotImplementedError("gradients in x, n and eps are stated for the dipole "
                                      "kernel only (channels with the foreshortening term)")

    def forward(self, queries, beta, counters=False):
        """PrimalQuery for every query (Alg. 1): [Q, C] float64 (and [Q,3] counters)."""
        if self.C is None:
            raise RuntimeError("call update() first")
        q = _f32(queries)
        nq = q.shape[0]
        out = np.zeros((nq, self.C), np.float64)
        cnt = np.zeros((nq, 3), np.int64) if counters else None
        _load().orc_bh_forward(self._h, nq, _ptr(q), float(beta), _ptr(out), _ptr(cnt))
        return (out, cnt) if counters else out

    def forward_bf16_allowance(self, queries, beta):
        """With bf16 moments (reading R13): the forward [Q, C] and, per query and
        channel, the bound on what roundings on the edge of a bf16 boundary can
        change (0 where no far node's sum is that close to one)."""
        if not getattr(self, "bf16_moments", False):
            raise RuntimeError("update(..., bf16_moments=True) first")
        q = _f32(queries)
        nq = q.shape[0]
        out = np.zeros((nq, self.C), np.float64)
        allow = np.zeros((nq, self.C), np.float64)
        _load().orc_bh_forward_bf16(self._h, nq, _ptr(q), float(beta), _ptr(out), None,
                                    _ptr(allow))
        return out, allow

    def near_ties(self, queries, beta):
        """Per query, the tested nodes whose double distance is within 1e-6 d of
        beta r~ (the far test's near ties, a diagnostic of reading R6): int64 [Q]."""
        q = _f32(queries)
        out = np.zeros(q.shape[0], np.int64)
        _load().orc_bh_near_ties(self._h, q.shape[0], _ptr(q), float(beta), _ptr(out))
        return out

    def forward_grad(self, queries, beta):
        """Barnes-Hut spatial gradient of the dipole sum: [Q, C, 3] float64."""
        if self.C is None:
            raise RuntimeError("call update() first")
        self._dipole_only()
        q = _f32(queries)
        out = np.zeros((q.shape[0], self.C, 3), np.float64)
        _load().orc_bh_forward_grad(self._h, q.shape[0], _ptr(q), float(beta), _ptr(out))
        return out

    def adjoint_grad(self, queries, beta, g=None, gg=None):
        """dL/dmu [N, C] for dL/dD = g [Q, C] and dL/d(grad D) = gg [Q, C, 3] (either may
        be None), two-stage (Sec. 6.2, App. C) extended to the gradient (R9)."""
        if self.C is None:
            raise RuntimeError("call update() first")
        self._dipole_only()
        q = _f32(queries)
        nq = q.shape[0]
        g64 = None if g is None else _f64(np.asarray(g).reshape(nq, self.C))
        gg64 = None if gg is None else _f64(np.asarray(gg).reshape(nq, self.C, 3))
        out = np.zeros((self.n, self.C), np.float64)
        _load().orc_bh_adjoint_grad(self._h, nq, _ptr(q), float(beta), _ptr(g64), _ptr(gg64),
                                    _ptr(out))
        return out

    def adjoint_geom(self, queries, beta, g=None, gg=None):
        """Barnes-Hut gradients of L(D, grad D) with respect to mu, the normals and
        eps (R10): (dmu [N, C], dn [N, 3], deps [N]) float64, input order."""
        if self.C is None:
            raise RuntimeError("call update() first")
        self._dipole_only()
        q = _f32(queries)
        nq = q.shape[0]
        g64 = None if g is None else _f64(np.asarray(g).reshape(nq, self.C))
        gg64 = None if gg is None else _f64(np.asarray(gg).reshape(nq, self.C, 3))
        dmu = np.zeros((self.n, self.C), np.float64)
        dn = np.zeros((self.n, 3), np.float64)
        deps = np.zeros(self.n, np.float64)
        _load().orc_bh_adjoint_geom(self._h, nq, _ptr(q), float(beta), _ptr(g64), _ptr(gg64),
                                    _ptr(dmu), _ptr(dn), _ptr(deps))
        return dmu, dn, deps

    def adjoint(self, queries, beta, g):
        """Two-stage adjoint (Sec. 6.2, App. C): dL/dmu [N, C] float64, input order."""
        if self.C is None:
            raise RuntimeError("call update() first")
        q = _f32(queries)
        g = _f64(g)
        if g.ndim == 1:
            g = g[:, None]
        if g.shape != (q.shape[0], self.C):
            raise ValueError("g must be [Q, C]")
        out = np.zeros((self.n, self.C), np.float64)
        _load().orc_bh_adjoint(self._h, q.shape[0], _ptr(q), float(beta), _ptr(g), _ptr(out))
        return out
