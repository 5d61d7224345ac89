"""CPU oracle for the dual-tree-traversal FMM (arXiv:1209.3516).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the
CPU-baseline leg of the benchmark may import this package; the GPU library
and its Python binding never do, and this package never imports them.

The arithmetic lives in ``fmm_oracle.c`` (plain C, FP64, OpenMP over targets).
This module only marshals NumPy arrays through ctypes.  Every function cites
the passage of the paper it follows in the C source.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(closed forms, brute force, exactness of re-expansion, convergence in P and
theta, exact reproduction of the direct sum at theta = 0, force balance and
the paper's Table 3 as a soft anchor).  The constants the paper does not give
(normalisation epsilon, split tie-break, degree convention, coincident
points) are readings, not pins.
"""
import ctypes
import os
import threading

import numpy as np

from .build import build_oracle

_lib = None
_lock = threading.Lock()

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i32p = ctypes.POINTER(ctypes.c_int32)


def lib():
    """Load (building if needed) the oracle shared library."""
    global _lib
    with _lock:
        if _lib is None:
            # ORC_LIB points at another build of fmm_oracle.c (the mutation
            # tests load deliberately broken copies through it)
            path = os.environ.get("ORC_LIB") or build_oracle()
            L = ctypes.CDLL(path)
            L.orc_nterms.argtypes = [ctypes.c_int]
            L.orc_nterms.restype = ctypes.c_int
            L.orc_multi_indices.argtypes = [ctypes.c_int, _i32p]
            L.orc_taylor.argtypes = [ctypes.c_int, _dp, _dp]
            for name in ("orc_m2m", "orc_m2l", "orc_l2l"):
                getattr(L, name).argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp]
                getattr(L, name).restype = ctypes.c_int
            L.orc_p2m.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
            L.orc_p2m.restype = ctypes.c_int
            L.orc_l2p.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, _dp, _dp, _dp]
            L.orc_l2p.restype = ctypes.c_int
            L.orc_direct.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_int64, _i64p, _dp, _dp]
            L.orc_direct_backward.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, ctypes.c_int64, _i64p,
                                              _dp, _dp]
            L.orc_p2m_dipole.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
            L.orc_p2m_dipole.restype = ctypes.c_int
            L.orc_l2p_hess.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
            L.orc_l2p_hess.restype = ctypes.c_int
            L.orc_morton.argtypes = [ctypes.c_uint32] * 3
            L.orc_morton.restype = ctypes.c_uint64
            L.orc_create.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_int]
            L.orc_create.restype = ctypes.c_void_p
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_build.argtypes = [ctypes.c_void_p, _dp]
            L.orc_build.restype = ctypes.c_int
            L.orc_evaluate.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int64, _i64p, _dp, _dp]
            L.orc_evaluate.restype = ctypes.c_int
            L.orc_backward.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, ctypes.c_int64, _i64p, _dp, _dp]
            L.orc_set_hybrid.argtypes = [ctypes.c_void_p, ctypes.c_int64]
            L.orc_backward.restype = ctypes.c_int
            for name in ("orc_ncells", "orc_nm2l", "orc_np2p"):
                getattr(L, name).argtypes = [ctypes.c_void_p]
                getattr(L, name).restype = ctypes.c_int64
            L.orc_norm.argtypes = [ctypes.c_void_p, _dp, _dp]
            L.orc_sorted.argtypes = [ctypes.c_void_p, _u64p, _i64p, _dp, _fp]
            L.orc_cells.argtypes = [ctypes.c_void_p, _u64p, _i32p, _i64p, _i64p, _i32p, _i64p,
                                    _fp, _fp]
            L.orc_lists.argtypes = [ctypes.c_void_p, _u64p, _u64p]
            L.orc_lists_idx.argtypes = [ctypes.c_void_p, _i64p, _i64p]
            L.orc_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def max_threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(lib().orc_max_threads())


def nterms(P: int) -> int:
    return int(lib().orc_nterms(P))


def multi_indices(P: int) -> np.ndarray:
    """(T, 3) table of the oracle's multi-index order."""
    T = nterms(P)
    k = np.zeros((T, 3), dtype=np.int32)
    lib().orc_multi_indices(P, _ptr(k, _i32p))
    return k


def taylor(P: int, R) -> np.ndarray:
    """Taylor coefficients b_m(R) = d^m(1/|R|)/m!, |m| <= P-1."""
    R = _f64(R, (3,))
    b = np.zeros(nterms(P))
    lib().orc_taylor(P, _ptr(R, _dp), _ptr(b, _dp))
    return b


def p2m(P, y, q, X):
    y = _f64(y, (-1, 3))
    q = _f64(q, (-1,))
    X = _f64(X, (3,))
    M = np.zeros(nterms(P))
    assert lib().orc_p2m(P, y.shape[0], _ptr(y, _dp), _ptr(q, _dp), _ptr(X, _dp), _ptr(M, _dp)) == 0
    return M


def m2m(P, Mc, Xc, Xp):
    Mc = _f64(Mc)
    Mp = np.zeros(nterms(P))
    assert lib().orc_m2m(P, _ptr(Mc, _dp), _ptr(_f64(Xc, (3,)), _dp), _ptr(_f64(Xp, (3,)), _dp),
                         _ptr(Mp, _dp)) == 0
    return Mp


def m2l(P, M, Xs, Xt):
    M = _f64(M)
    L = np.zeros(nterms(P))
    assert lib().orc_m2l(P, _ptr(M, _dp), _ptr(_f64(Xs, (3,)), _dp), _ptr(_f64(Xt, (3,)), _dp),
                         _ptr(L, _dp)) == 0
    return L


def l2l(P, Lp, Xp, Xc):
    Lp = _f64(Lp)
    Lc = np.zeros(nterms(P))
    assert lib().orc_l2l(P, _ptr(Lp, _dp), _ptr(_f64(Xp, (3,)), _dp), _ptr(_f64(Xc, (3,)), _dp),
                         _ptr(Lc, _dp)) == 0
    return Lc


def l2p(P, L, Xt, x):
    L = _f64(L)
    x = _f64(x, (-1, 3))
    phi = np.zeros(x.shape[0])
    grad = np.zeros((x.shape[0], 3))
    assert lib().orc_l2p(P, _ptr(L, _dp), _ptr(_f64(Xt, (3,)), _dp), x.shape[0], _ptr(x, _dp),
                         _ptr(phi, _dp), _ptr(grad, _dp)) == 0
    return phi, grad


def p2m_dipole(P, y, a, p, X):
    """Multipole of sources with charges a and dipoles p (n x 3) about X."""
    y = _f64(y, (-1, 3))
    a = _f64(a, (-1,))
    p = _f64(p, (-1, 3))
    M = np.zeros(nterms(P))
    assert lib().orc_p2m_dipole(P, y.shape[0], _ptr(y, _dp), _ptr(a, _dp), _ptr(p, _dp),
                                _ptr(_f64(X, (3,)), _dp), _ptr(M, _dp)) == 0
    return M


def l2p_hess(P, L, Xt, x, v):
    """Hessian of the local expansion L (about Xt) at x, applied to v."""
    hv = np.zeros(3)
    assert lib().orc_l2p_hess(P, _ptr(_f64(L), _dp), _ptr(_f64(Xt, (3,)), _dp), _ptr(_f64(x, (3,)), _dp),
                              _ptr(_f64(v, (3,)), _dp), _ptr(hv, _dp)) == 0
    return hv


def morton(ix: int, iy: int, iz: int) -> int:
    return int(lib().orc_morton(ix, iy, iz))


def direct(x, q, targets=None):
    """FP64 direct sum: phi_i = sum_j q_j/r_ij, grad_i = -sum_j q_j (x_i-x_j)/r_ij^3."""
    x = _f64(x, (-1, 3))
    q = _f64(q, (-1,))
    N = x.shape[0]
    if targets is None:
        nt, tp = N, None
    else:
        t = np.ascontiguousarray(targets, dtype=np.int64)
        nt, tp = t.shape[0], t
    phi = np.zeros(nt)
    grad = np.zeros((nt, 3))
    lib().orc_direct(N, _ptr(x, _dp), _ptr(q, _dp), nt if tp is not None else 0,
                     _ptr(tp, _i64p), _ptr(phi, _dp), _ptr(grad, _dp))
    return phi, grad


def direct_backward(x, q, dphi=None, dgrad=None, targets=None):
    """FP64 adjoint of the direct sum: (dL/dq, dL/dx) for upstream dL/dphi, dL/dgrad."""
    x = _f64(x, (-1, 3))
    q = _f64(q, (-1,))
    N = x.shape[0]
    a = None if dphi is None else _f64(dphi, (N,))
    b = None if dgrad is None else _f64(dgrad, (N, 3))
    if targets is None:
        nt, tp = N, None
    else:
        tp = np.ascontiguousarray(targets, dtype=np.int64)
        nt = tp.shape[0]
    dq = np.zeros(nt)
    dx = np.zeros((nt, 3))
    lib().orc_direct_backward(N, _ptr(x, _dp), _ptr(q, _dp), _ptr(a, _dp), _ptr(b, _dp),
                              nt if tp is not None else 0, _ptr(tp, _i64p), _ptr(dq, _dp), _ptr(dx, _dp))
    return dq, dx


class FMM:
    """Oracle FMM: tree + dual tree traversal + FP64 Cartesian Taylor evaluation."""

    def __init__(self, N: int, P: int, theta: float, ncrit: int, hybrid_min_pairs: int = -1):
        self._h = lib().orc_create(int(N), int(P), float(theta), int(ncrit))
        if not self._h:
            raise ValueError("oracle rejected N=%r P=%r theta=%r ncrit=%r" % (N, P, theta, ncrit))
        self.N, self.P, self.theta, self.ncrit = int(N), int(P), float(theta), int(ncrit)
        # the M2L / P2P hybrid at the leaves (-1: Algorithm 4 as printed)
        lib().orc_set_hybrid(self._h, int(hybrid_min_pairs))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def build(self, x):
        x = _f64(x, (self.N, 3))
        rc = lib().orc_build(self._h, _ptr(x, _dp))
        if rc != 0:
            raise ValueError("oracle build failed (non-finite input or out of memory)")
        return self

    def evaluate(self, q, targets=None):
        q = _f64(q, (self.N,))
        if targets is None:
            nt, tp = self.N, None
        else:
            tp = np.ascontiguousarray(targets, dtype=np.int64)
            nt = tp.shape[0]
        phi = np.zeros(nt)
        grad = np.zeros((nt, 3))
        rc = lib().orc_evaluate(self._h, _ptr(q, _dp), nt if tp is not None else 0,
                                _ptr(tp, _i64p), _ptr(phi, _dp), _ptr(grad, _dp))
        if rc != 0:
            raise ValueError("oracle evaluate failed")
        return phi, grad

    def backward(self, q, dphi=None, dgrad=None, targets=None):
        """FMM adjoint: (dL/dq, dL/dx) for charges q and upstream dL/dphi, dL/dgrad."""
        q = _f64(q, (self.N,))
        a = None if dphi is None else _f64(dphi, (self.N,))
        b = None if dgrad is None else _f64(dgrad, (self.N, 3))
        if targets is None:
            nt, tp = self.N, None
        else:
            tp = np.ascontiguousarray(targets, dtype=np.int64)
            nt = tp.shape[0]
        dq = np.zeros(nt)
        dx = np.zeros((nt, 3))
        rc = lib().orc_backward(self._h, _ptr(q, _dp), _ptr(a, _dp), _ptr(b, _dp), nt if tp is not None else 0,
                                _ptr(tp, _i64p), _ptr(dq, _dp), _ptr(dx, _dp))
        if rc != 0:
            raise ValueError("oracle backward failed")
        return dq, dx

    @property
    def ncells(self) -> int:
        return int(lib().orc_ncells(self._h))

    def norm(self):
        c = np.zeros(3)
        h = np.zeros(1)
        lib().orc_norm(self._h, _ptr(c, _dp), _ptr(h, _dp))
        return c, float(h[0])

    def sorted(self):
        N = self.N
        key = np.zeros(N, dtype=np.uint64)
        perm = np.zeros(N, dtype=np.int64)
        u = np.zeros((N, 3))
        u32 = np.zeros((N, 3), dtype=np.float32)
        lib().orc_sorted(self._h, _ptr(key, _u64p), _ptr(perm, _i64p), _ptr(u, _dp), _ptr(u32, _fp))
        return {"key": key, "perm": perm, "u": u, "u32": u32}

    def cells(self):
        n = self.ncells
        out = {
            "canon": np.zeros(n, dtype=np.uint64),
            "level": np.zeros(n, dtype=np.int32),
            "pbeg": np.zeros(n, dtype=np.int64),
            "pcnt": np.zeros(n, dtype=np.int64),
            "nchild": np.zeros(n, dtype=np.int32),
            "parent": np.zeros(n, dtype=np.int64),
            "centre": np.zeros((n, 3), dtype=np.float32),
            "radius": np.zeros(n, dtype=np.float32),
        }
        lib().orc_cells(self._h, _ptr(out["canon"], _u64p), _ptr(out["level"], _i32p),
                        _ptr(out["pbeg"], _i64p), _ptr(out["pcnt"], _i64p),
                        _ptr(out["nchild"], _i32p), _ptr(out["parent"], _i64p),
                        _ptr(out["centre"], _fp), _ptr(out["radius"], _fp))
        return out

    def lists(self):
        """(m2l, p2p) as (n, 2) uint64 arrays of canonical (target, source) cell ids."""
        nm = int(lib().orc_nm2l(self._h))
        npp = int(lib().orc_np2p(self._h))
        m = np.zeros((nm, 2), dtype=np.uint64)
        p = np.zeros((npp, 2), dtype=np.uint64)
        lib().orc_lists(self._h, _ptr(m, _u64p), _ptr(p, _u64p))
        return m, p

    def lists_idx(self):
        """(m2l, p2p) as (n, 2) int64 arrays of cell indices (into cells())."""
        nm = int(lib().orc_nm2l(self._h))
        npp = int(lib().orc_np2p(self._h))
        m = np.zeros((nm, 2), dtype=np.int64)
        p = np.zeros((npp, 2), dtype=np.int64)
        lib().orc_lists_idx(self._h, _ptr(m, _i64p), _ptr(p, _i64p))
        return m, p
