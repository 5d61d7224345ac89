"""Thin Python binding of the C-ABI library (include/fmm.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides device memory and the stream.  The library is
built in-tree by ``paper_1209_3516_gb300.build.build()``; if it is missing
this module raises instead of falling back to anything else.
"""
import ctypes
import os

import numpy as np

from . import build as _build

FMM_OK = 0
FMM_ERR_ARG = -1
FMM_ERR_UNSUPPORTED = -2
FMM_ERR_INPUT = -3
FMM_ERR_CUDA = -4
FMM_ERR_NOMEM = -5
FMM_ERR_STATE = -6
FMM_ERR_CAPACITY = -7

FMM_FLAG_KAHAN = 1
FMM_FLAG_TIMING = 2
FMM_FLAG_MUTUAL = 4

PHASES = ["morton", "sort", "tree", "traverse", "lists", "items", "upward", "m2l", "downward", "p2p"]


class FMMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (code %d)" % (msg, code))
        self.code = code


class _Options(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("device", ctypes.c_int), ("flags", ctypes.c_uint)]


class _Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ncells", ctypes.c_int64), ("nleaves", ctypes.c_int64),
                ("nlevels", ctypes.c_int32), ("P", ctypes.c_int32), ("n_m2l", ctypes.c_int64),
                ("n_p2p", ctypes.c_int64), ("p2p_pairs", ctypes.c_int64), ("ms_build", ctypes.c_double),
                ("ms_evaluate", ctypes.c_double), ("ms_phase", ctypes.c_double * len(PHASES)),
                ("kernel_launches", ctypes.c_int64), ("ms_backward", ctypes.c_double),
                ("ms_batch", ctypes.c_double)]

MAX_RHS = 32


class _Peaks(ctypes.Structure):
    _fields_ = [("ffma_tflops", ctypes.c_double), ("ffma2_tflops", ctypes.c_double), ("rsqrt_per_s", ctypes.c_double),
                ("ms_ffma", ctypes.c_double), ("ms_ffma2", ctypes.c_double), ("ms_rsqrt", ctypes.c_double),
                ("sms", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _MultiInfo(ctypes.Structure):
    _fields_ = [("n_total", ctypes.c_int64), ("ncells", ctypes.c_int64), ("nleaves", ctypes.c_int64),
                ("n_m2l", ctypes.c_int64), ("p2p_pairs", ctypes.c_int64), ("graph_nodes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("nsys", ctypes.c_int32), ("nlevels", ctypes.c_int32),
                ("p2p_targets_per_item", ctypes.c_int32), ("mutual", ctypes.c_int32),
                ("tune_ms", ctypes.c_double * 6), ("ms_evaluate", ctypes.c_double)]


_lib = None
_vp = ctypes.c_void_p


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libfmm_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError("libfmm_gb300.so is not built (%s); run __graft_entry__.build() or "
                           "python -m paper_1209_3516_gb300.build" % path)
    L = ctypes.CDLL(path)
    L.fmm_last_error_string.restype = ctypes.c_char_p
    L.fmm_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                             ctypes.POINTER(_Options)]
    L.fmm_build.argtypes = [_vp, _vp]
    L.fmm_evaluate.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.fmm_evaluate_host.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.fmm_evaluate_batch.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, _vp]
    L.fmm_energy.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
    L.fmm_backward.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.fmm_stats.argtypes = [_vp, ctypes.POINTER(_Stats)]
    L.fmm_destroy.argtypes = [_vp]
    L.fmm_get_norm.argtypes = [_vp, _vp, _vp]
    L.fmm_get_sorted.argtypes = [_vp, _vp, _vp]
    L.fmm_get_ncells.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
    L.fmm_get_cells.argtypes = [_vp] + [_vp] * 8
    L.fmm_get_lists.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), _vp, _vp]
    L.fmm_energy_noalloc.argtypes = [_vp, _vp, ctypes.c_int64, _vp, _vp]
    L.fmm_measure_peaks.argtypes = [ctypes.POINTER(_Peaks), _vp]
    L.fmm_multi_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                   ctypes.c_float, ctypes.c_int, ctypes.POINTER(_Options)]
    L.fmm_multi_build.argtypes = [_vp, _vp]
    L.fmm_multi_evaluate.argtypes = [_vp, _vp, _vp, _vp]
    L.fmm_multi_info.argtypes = [_vp, ctypes.POINTER(_MultiInfo)]
    L.fmm_multi_destroy.argtypes = [_vp]
    L.fmm_multi_set_hybrid.argtypes = [_vp, ctypes.c_int64]
    L.fmm_multi_set_config.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
    L.fmm_set_hybrid.argtypes = [_vp, ctypes.c_int64]
    L.fmm_tune_hybrid.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_int, _vp, _vp,
                                  ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_int, ctypes.POINTER(_Options),
                                  ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
    L.fmm_tune_ncrit.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_float, _vp, _vp, ctypes.POINTER(ctypes.c_int),
                                 ctypes.c_int, ctypes.c_int, ctypes.POINTER(_Options), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_double)]
    _lib = L
    return L


def _check(rc):
    if rc != FMM_OK:
        raise FMMError(rc, load().fmm_last_error_string().decode())


def _np_ptr(a):
    return a.ctypes.data if a is not None else None


def _dev_ptr(t, dtype, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError("%s must be contiguous with shape %s, got %s" % (name, shape, tuple(t.shape)))
    return t.data_ptr()


def tune_ncrit(x, q, P, theta, candidates=(16, 32, 48, 64, 96, 128), reps=3, stream=None):
    """fmm_tune_ncrit: (best ncrit, {ncrit: median ms of build + evaluate})."""
    import torch
    N = x.shape[0]
    xp = _dev_ptr(x, torch.float64, (N, 3), "x")
    qp = _dev_ptr(q, torch.float32, (N,), "q")
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    opt = _Options(ctypes.c_void_p(stream.cuda_stream), x.device.index or 0, 0)
    cand = (ctypes.c_int * len(candidates))(*candidates)
    ms = (ctypes.c_double * len(candidates))()
    best = ctypes.c_int()
    _check(load().fmm_tune_ncrit(N, int(P), float(theta), xp, qp, cand, len(candidates), int(reps),
                                 ctypes.byref(opt), ctypes.byref(best), ms))
    return best.value, {c: ms[i] for i, c in enumerate(candidates)}


def tune_hybrid(x, q, P, theta, ncrit=64, candidates=(-1, 0, 256, 512, 1024, 2048), reps=3, stream=None):
    """fmm_tune_hybrid: (best min_pairs, {min_pairs: median ms of build + evaluate}); -1 = Algorithm 4."""
    import torch
    N = x.shape[0]
    xp = _dev_ptr(x, torch.float64, (N, 3), "x")
    qp = _dev_ptr(q, torch.float32, (N,), "q")
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    opt = _Options(ctypes.c_void_p(stream.cuda_stream), x.device.index or 0, 0)
    cand = (ctypes.c_int64 * len(candidates))(*candidates)
    ms = (ctypes.c_double * len(candidates))()
    best = ctypes.c_int64()
    _check(load().fmm_tune_hybrid(N, int(P), float(theta), int(ncrit), xp, qp, cand, len(candidates), int(reps),
                                  ctypes.byref(opt), ctypes.byref(best), ms))
    return best.value, {c: ms[i] for i, c in enumerate(candidates)}


def measure_peaks(stream=None):
    """fmm_measure_peaks on the current device: FP32 FFMA / FFMA2 TFLOP/s and SFU rsqrt/s, measured."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    pk = _Peaks()
    _check(load().fmm_measure_peaks(ctypes.byref(pk), ctypes.c_void_p(stream.cuda_stream)))
    return {f: getattr(pk, f) for f, _ in _Peaks._fields_ if f != "reserved"}


def energy_noalloc(q, phi, E, stream=None):
    """fmm_energy_noalloc: E[0] = 1/2 sum q phi into the caller's device double E (no allocation).

    q, phi and E must sit on one CUDA device; the call runs with that device current."""
    import torch
    n = q.numel()
    devs = {t.device for t in (q, phi, E)}
    if len(devs) != 1 or q.device.type != "cuda":
        raise ValueError("energy_noalloc: q, phi and E must be on one CUDA device (got %s)" % sorted(map(str, devs)))
    with torch.cuda.device(q.device):
        qp = _dev_ptr(q, torch.float32, (n,), "q")
        pp = _dev_ptr(phi, torch.float32, (n,), "phi")
        ep = _dev_ptr(E, torch.float64, (1,), "E")
        if stream is None:
            stream = torch.cuda.current_stream(q.device)
        _check(load().fmm_energy_noalloc(qp, pp, n, ep, ctypes.c_void_p(stream.cuda_stream)))
    return E


class FMM:
    """A handle: fmm_create(N, P, theta, ncrit) on the current CUDA device and stream."""

    def __init__(self, N, P=4, theta=0.4, ncrit=64, kahan=False, timing=False, stream=None, device=None,
                 hybrid=None, mutual=False):
        import torch
        L = load()
        if device is None:
            device = torch.cuda.current_device()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self.device = int(device)
        opt = _Options(ctypes.c_void_p(stream.cuda_stream), self.device,
                       (FMM_FLAG_KAHAN if kahan else 0) | (FMM_FLAG_TIMING if timing else 0) |
                       (FMM_FLAG_MUTUAL if mutual else 0))
        h = _vp()
        _check(L.fmm_create(ctypes.byref(h), int(N), int(P), float(theta), int(ncrit), ctypes.byref(opt)))
        self._h = h
        self.N, self.P, self.theta, self.ncrit = int(N), int(P), float(theta), int(ncrit)
        if hybrid is not None:   # M2L / P2P hybrid at the leaves: minimum particle pairs for M2L
            _check(L.fmm_set_hybrid(h, int(hybrid)))
        self.evaluations = 0   # fmm_evaluate calls so far (the adjoint differentiates the last one)

    def close(self):
        if getattr(self, "_h", None):
            load().fmm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- compute ----
    def build(self, x):
        import torch
        _check(load().fmm_build(self._h, _dev_ptr(x, torch.float64, (self.N, 3), "x")))
        return self

    def evaluate(self, q, x=None, phi=None, grad=None, want_phi=True, want_grad=True):
        """Potential (N,) and gradient (N, 3) as float32 CUDA tensors (caller order)."""
        import torch
        dev = torch.device("cuda", self.device)
        qp = _dev_ptr(q, torch.float32, (self.N,), "q")
        xp = _dev_ptr(x, torch.float64, (self.N, 3), "x") if x is not None else None
        if want_phi and phi is None:
            phi = torch.empty(self.N, dtype=torch.float32, device=dev)
        if want_grad and grad is None:
            grad = torch.empty(self.N, 3, dtype=torch.float32, device=dev)
        pp = _dev_ptr(phi, torch.float32, (self.N,), "phi") if phi is not None else None
        gp = _dev_ptr(grad, torch.float32, (self.N, 3), "grad") if grad is not None else None
        _check(load().fmm_evaluate(self._h, xp, qp, pp, gp))
        self.evaluations += 1
        return phi, grad

    def evaluate_batch(self, q, x=None, phi=None, grad=None, want_phi=True, want_grad=True):
        """fmm_evaluate_batch: q (nrhs, N) float32 CUDA -> phi (nrhs, N), grad (nrhs, N, 3)."""
        import torch
        dev = torch.device("cuda", self.device)
        if q.dim() != 2:
            raise ValueError("q must be (nrhs, N)")
        nrhs = q.shape[0]
        qp = _dev_ptr(q, torch.float32, (nrhs, self.N), "q")
        xp = _dev_ptr(x, torch.float64, (self.N, 3), "x") if x is not None else None
        if want_phi and phi is None:
            phi = torch.empty(nrhs, self.N, dtype=torch.float32, device=dev)
        if want_grad and grad is None:
            grad = torch.empty(nrhs, self.N, 3, dtype=torch.float32, device=dev)
        pp = _dev_ptr(phi, torch.float32, (nrhs, self.N), "phi") if phi is not None else None
        gp = _dev_ptr(grad, torch.float32, (nrhs, self.N, 3), "grad") if grad is not None else None
        _check(load().fmm_evaluate_batch(self._h, xp, qp, int(nrhs), pp, gp))
        return phi, grad

    def evaluate_host(self, x, q, phi=None, grad=None):
        """Host-buffer path: NumPy in, NumPy out (copies inside the library)."""
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.N, 3)
        q = np.ascontiguousarray(q, dtype=np.float32).reshape(self.N)
        if phi is None:
            phi = np.empty(self.N, dtype=np.float32)
        if grad is None:
            grad = np.empty((self.N, 3), dtype=np.float32)
        _check(load().fmm_evaluate_host(self._h, _np_ptr(x), _np_ptr(q), _np_ptr(phi), _np_ptr(grad)))
        self.evaluations += 1
        return phi, grad

    def energy(self) -> float:
        E = ctypes.c_double()
        _check(load().fmm_energy(self._h, ctypes.byref(E)))
        return E.value

    def backward(self, dphi=None, dgrad=None, dq=None, dx=None, want_dq=True, want_dx=True):
        """fmm_backward: (dL/dq (N,), dL/dx (N, 3)) float32 CUDA tensors for the
        upstream gradients dphi (N,) and dgrad (N, 3) of the last evaluate."""
        import torch
        dev = torch.device("cuda", self.device)
        if want_dq and dq is None:
            dq = torch.empty(self.N, dtype=torch.float32, device=dev)
        if want_dx and dx is None:
            dx = torch.empty(self.N, 3, dtype=torch.float32, device=dev)
        pp = _dev_ptr(dphi, torch.float32, (self.N,), "dphi") if dphi is not None else None
        gp = _dev_ptr(dgrad, torch.float32, (self.N, 3), "dgrad") if dgrad is not None else None
        qp = _dev_ptr(dq, torch.float32, (self.N,), "dq") if dq is not None else None
        xp = _dev_ptr(dx, torch.float32, (self.N, 3), "dx") if dx is not None else None
        _check(load().fmm_backward(self._h, pp, gp, qp, xp))
        return dq, dx

    # ---- counters / introspection ----
    def stats(self) -> dict:
        s = _Stats()
        _check(load().fmm_stats(self._h, ctypes.byref(s)))
        d = {k: getattr(s, k) for k, _ in _Stats._fields_ if k != "ms_phase"}
        d["ms_phase"] = {name: s.ms_phase[i] for i, name in enumerate(PHASES)}
        return d

    def norm(self):
        c = np.zeros(3)
        h = np.zeros(1)
        _check(load().fmm_get_norm(self._h, _np_ptr(c), _np_ptr(h)))
        return c, float(h[0])

    def sorted(self):
        keys = np.zeros(self.N, dtype=np.uint64)
        perm = np.zeros(self.N, dtype=np.int32)
        _check(load().fmm_get_sorted(self._h, _np_ptr(keys), _np_ptr(perm)))
        return keys, perm

    def ncells(self) -> int:
        n = ctypes.c_int64()
        _check(load().fmm_get_ncells(self._h, ctypes.byref(n)))
        return n.value

    def cells(self) -> dict:
        n = self.ncells()
        out = {"canon": np.zeros(n, dtype=np.uint64), "level": np.zeros(n, dtype=np.int32),
               "pbeg": np.zeros(n, dtype=np.int32), "pcnt": np.zeros(n, dtype=np.int32),
               "nchild": np.zeros(n, dtype=np.int32), "parent": np.zeros(n, dtype=np.int32),
               "centre": np.zeros((n, 3), dtype=np.float32), "radius": np.zeros(n, dtype=np.float32)}
        _check(load().fmm_get_cells(self._h, *[_np_ptr(out[k]) for k in
                                               ("canon", "level", "pbeg", "pcnt", "nchild", "parent", "centre",
                                                "radius")]))
        return out

    def lists(self, fetch=True):
        """(m2l, p2p) as (n, 2) int32 (target, source) cell indices, grouped and sorted."""
        nm, npp = ctypes.c_int64(), ctypes.c_int64()
        _check(load().fmm_get_lists(self._h, ctypes.byref(nm), ctypes.byref(npp), None, None))
        if not fetch:
            return nm.value, npp.value
        m = np.zeros((nm.value, 2), dtype=np.int32)
        p = np.zeros((npp.value, 2), dtype=np.int32)
        _check(load().fmm_get_lists(self._h, None, None, _np_ptr(m), _np_ptr(p)))
        return m, p


class MultiFMM:
    """fmm_multi_*: many independent systems (sizes N[s]) evaluated as one merged
    problem, replayed from a CUDA graph."""

    def __init__(self, sizes, P=4, theta=0.4, ncrit=64, stream=None, device=None, hybrid=None):
        import torch
        L = load()
        if device is None:
            device = torch.cuda.current_device()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream, self.device = stream, int(device)
        self.sizes = [int(n) for n in sizes]
        self.N = sum(self.sizes)
        arr = (ctypes.c_int64 * len(self.sizes))(*self.sizes)
        opt = _Options(ctypes.c_void_p(stream.cuda_stream), self.device, 0)
        h = _vp()
        _check(L.fmm_multi_create(ctypes.byref(h), len(self.sizes), arr, int(P), float(theta), int(ncrit),
                                  ctypes.byref(opt)))
        self._h = h
        if hybrid is not None:
            _check(L.fmm_multi_set_hybrid(h, int(hybrid)))

    def close(self):
        if getattr(self, "_h", None):
            load().fmm_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build(self, x):
        import torch
        _check(load().fmm_multi_build(self._h, _dev_ptr(x, torch.float64, (self.N, 3), "x")))
        return self

    def evaluate(self, q, phi=None, grad=None):
        import torch
        dev = torch.device("cuda", self.device)
        qp = _dev_ptr(q, torch.float32, (self.N,), "q")
        if phi is None:
            phi = torch.empty(self.N, dtype=torch.float32, device=dev)
        if grad is None:
            grad = torch.empty(self.N, 3, dtype=torch.float32, device=dev)
        _check(load().fmm_multi_evaluate(self._h, qp, _dev_ptr(phi, torch.float32, (self.N,), "phi"),
                                         _dev_ptr(grad, torch.float32, (self.N, 3), "grad")))
        return phi, grad

    def set_config(self, targets_per_item=0, mutual=-1):
        """fmm_multi_set_config: pin the near field (0 / -1 let the autotuner choose; mutual 0 one-sided,
        1 / 2 mutual with 2 / 4 staged sources per lane)."""
        _check(load().fmm_multi_set_config(self._h, int(targets_per_item), int(mutual)))

    def info(self) -> dict:
        i = _MultiInfo()
        _check(load().fmm_multi_info(self._h, ctypes.byref(i)))
        d = {k: getattr(i, k) for k, _ in _MultiInfo._fields_ if k not in ("tune_ms", "reserved")}
        d["tune_ms"] = [i.tune_ms[k] for k in range(6)]
        return d
