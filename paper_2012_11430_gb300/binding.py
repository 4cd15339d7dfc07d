"""ctypes binding of the C ABI in include/prony.h (argument marshalling only).

Every computation happens in libprony.so; this module converts numpy arrays and
torch tensors to pointers and sizes and back.  If the library has not been built
(or fails to load) every call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libprony.so")

PRONY_OK, PRONY_EINVAL, PRONY_ERANK, PRONY_ENOCONV, PRONY_ENAN, PRONY_ECUDA, PRONY_ENOMEM = 0, -1, -2, -3, -4, -5, -6
PRONY_FP32, PRONY_BF16X3, PRONY_TF32X3, PRONY_BF16X2, PRONY_FFT32 = 0, 1, 2, 3, 4
PRECISIONS = {"fp32": PRONY_FP32, "bf16x3": PRONY_BF16X3, "tf32x3": PRONY_TF32X3, "bf16x2": PRONY_BF16X2,
              "fft32": PRONY_FFT32}

EXPORTS = [
    "prony_default_opts", "prony_status_string", "prony_last_error", "prony_ctx_create", "prony_ctx_destroy",
    "prony_solve", "prony_build_S", "prony_eval", "prony_solve_batched", "prony_solve_batched_dev",
    "prony_expsum_fwd_dev", "prony_expsum_bwd_dev", "prony_toeplitz_mm_dev", "prony_set_profiling",
    "prony_get_stats", "prony_toeplitz_mm_static", "prony_refine_lm_dev", "prony_small_steps",
]


class PronyStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("toeplitz_launches", ctypes.c_longlong),
                ("toeplitz_ms", ctypes.c_double), ("toeplitz_flops", ctypes.c_double),
                ("toeplitz_bytes", ctypes.c_double), ("tc_ksplit", ctypes.c_int),
                ("tc_bstages", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PronyOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("oversample_p", ctypes.c_int), ("tol_rank", ctypes.c_double),
                ("tol_power", ctypes.c_double), ("max_iter", ctypes.c_int), ("seed", ctypes.c_ulonglong),
                ("rank_mode", ctypes.c_int), ("vandermonde", ctypes.c_int), ("svd_method", ctypes.c_int)]


class PronyInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("rank_detected", ctypes.c_int), ("rank_used", ctypes.c_int),
                ("power_iters", ctypes.c_int), ("power_resid", ctypes.c_double), ("ls_resid", ctypes.c_double),
                ("sigma_ratio", ctypes.c_double), ("normT", ctypes.c_double), ("lanczos_steps", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PronyError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: status {code} ({status_string(code)}) {last_error()}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libprony.so (raises OSError / FileNotFoundError when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} not built; run paper_2012_11430_gb300/build.py")
    lib = ctypes.CDLL(path)
    P, I, D, LL, ULL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_ulonglong
    lib.prony_default_opts.argtypes = [ctypes.POINTER(PronyOpts)]
    lib.prony_default_opts.restype = None
    lib.prony_status_string.argtypes = [I]
    lib.prony_status_string.restype = ctypes.c_char_p
    lib.prony_last_error.argtypes = []
    lib.prony_last_error.restype = ctypes.c_char_p
    lib.prony_ctx_create.argtypes = [ctypes.POINTER(P), I]
    lib.prony_ctx_destroy.argtypes = [P]
    lib.prony_solve.argtypes = [P, P, I, I, I, P, P, P, P]
    lib.prony_build_S.argtypes = [P, P, I, I, I, P, P, P, P, P, P]
    lib.prony_eval.argtypes = [P, P, P, I, I, P, I, P]
    lib.prony_solve_batched.argtypes = [P, I, P, P, P, P, P, P, P, P, P, P]
    lib.prony_solve_batched_dev.argtypes = [P, I, P, P, P, P, P, P, P, P, P, P, P]
    lib.prony_expsum_fwd_dev.argtypes = [P, P, P, I, I, P, P, P, P]
    lib.prony_expsum_bwd_dev.argtypes = [P, P, P, I, I, P, P, P, P, P, P]
    lib.prony_refine_lm_dev.argtypes = [P, P, P, I, I, P, P, P, I, ctypes.c_double, P, P]
    lib.prony_toeplitz_mm_dev.argtypes = [P, P, I, I, P, I, I, I, I, P, P]
    lib.prony_toeplitz_mm_static.argtypes = [P, I, I, P, I, I, I, P, P]
    lib.prony_set_profiling.argtypes = [P, I]
    lib.prony_get_stats.argtypes = [P, ctypes.POINTER(PronyStats)]
    lib.prony_small_steps.argtypes = [P, I, I, I, P, P, ULL, I, I, P, P, P, P, P]
    for name in EXPORTS:
        if name not in ("prony_default_opts", "prony_status_string", "prony_last_error"):
            getattr(lib, name).restype = I
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().prony_status_string(code).decode()


def last_error() -> str:
    return load().prony_last_error().decode()


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def toeplitz_mm_static(grid_dev, d: int, n: int, X_dev, L: int, adjoint: int, Y_dev, stream: int = 0) -> int:
    """Allocation-free Toeplitz product on the current device (asynchronous on `stream`).

    For callers that cannot let the library allocate device memory; it needs no Context.
    Scratch lives in a fixed device array shared by all calls (overlapping calls race)."""
    r = X_dev.shape[0] if X_dev.dim() == 2 else 1
    rc = load().prony_toeplitz_mm_static(ctypes.c_void_p(grid_dev.data_ptr()), d, n,
                                         ctypes.c_void_p(X_dev.data_ptr()), r, L, adjoint,
                                         ctypes.c_void_p(Y_dev.data_ptr()), ctypes.c_void_p(stream))
    return _check(rc, "prony_toeplitz_mm_static")


def default_opts(**kw) -> PronyOpts:
    o = PronyOpts()
    load().prony_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        setattr(o, k, v)
    return o


def _check(rc: int, what: str, allow=(PRONY_OK,)):
    if rc not in allow:
        raise PronyError(rc, what)
    return rc


def _grid_c128(grid: np.ndarray, d: int, n: int) -> np.ndarray:
    g = np.ascontiguousarray(grid, dtype=np.complex128)
    if g.size != (2 * n + 2) ** d:
        raise ValueError("grid must hold (2n+2)^d samples")
    return g


@dataclass
class SolveResult:
    t: np.ndarray
    c: np.ndarray
    info: dict


class Context:
    """A library context on one CUDA device (owns the device workspace and a stream)."""

    def __init__(self, device: int = 0):
        self._lib = load()
        self._h = ctypes.c_void_p()
        _check(self._lib.prony_ctx_create(ctypes.byref(self._h), device), "prony_ctx_create")

    def close(self):
        if self._h:
            self._lib.prony_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_profiling(self, enable: bool = True):
        _check(self._lib.prony_set_profiling(self._h, int(enable)), "prony_set_profiling")

    def stats(self) -> dict:
        s = PronyStats()
        _check(self._lib.prony_get_stats(self._h, ctypes.byref(s)), "prony_get_stats")
        return s.as_dict()

    # ---------------------------------------------------------------- host-pointer calls
    def solve(self, grid, d: int, n: int, m: int, opts: PronyOpts | None = None,
              allow=(PRONY_OK, PRONY_ERANK)) -> SolveResult:
        g = _grid_c128(grid, d, n)
        t = np.zeros((m, d))
        c = np.zeros(m, dtype=np.complex128)
        info = PronyInfo()
        rc = self._lib.prony_solve(self._h, _ptr(g), d, n, m, ctypes.byref(opts) if opts else None,
                                   _ptr(t), _ptr(c), ctypes.byref(info))
        _check(rc, "prony_solve", allow)
        return SolveResult(t, c, info.as_dict())

    def build_S(self, grid, d: int, n: int, m: int, opts: PronyOpts | None = None, want_uv: bool = False,
                allow=(PRONY_OK, PRONY_ERANK)):
        g = _grid_c128(grid, d, n)
        N = (n + 1) ** d
        S = np.zeros((d, m, m), dtype=np.complex128)
        sig = np.zeros(m)
        U = np.zeros((m, N), dtype=np.complex128) if want_uv else None
        V = np.zeros((m, N), dtype=np.complex128) if want_uv else None
        info = PronyInfo()
        rc = self._lib.prony_build_S(self._h, _ptr(g), d, n, m, ctypes.byref(opts) if opts else None, _ptr(S),
                                     _ptr(sig), _ptr(U) if want_uv else None, _ptr(V) if want_uv else None,
                                     ctypes.byref(info))
        _check(rc, "prony_build_S", allow)
        # column-major N x m on the C side == row-major m x N here
        return S, sig, (U.T.copy() if want_uv else None), (V.T.copy() if want_uv else None), info.as_dict()

    def small_steps(self, Q, M, seed: int = 1, jacobi_cap: int = 0, eigqr_cap: int = 0):
        """The FP64 steps after the products on given Q (a x m) and M (d, a, m): returns
        (sigma, S (d, m, m), z (m, d), t (m, d), status)."""
        Q = np.ascontiguousarray(Q, dtype=np.complex128)
        M = np.ascontiguousarray(M, dtype=np.complex128)
        a, m = Q.shape
        d = M.shape[0]
        if M.shape != (d, a, m):
            raise ValueError("M must be (d, a, m)")
        sig = np.zeros(m)
        S = np.zeros((d, m, m), dtype=np.complex128)
        z = np.zeros((m, d), dtype=np.complex128)
        t = np.zeros((m, d))
        st = ctypes.c_int(0)
        _check(self._lib.prony_small_steps(self._h, d, m, a, _ptr(Q), _ptr(M), ctypes.c_ulonglong(seed),
                                           int(jacobi_cap), int(eigqr_cap), _ptr(sig), _ptr(S), _ptr(z), _ptr(t),
                                           ctypes.byref(st)), "prony_small_steps")
        return sig, S, z, t, st.value

    def eval(self, t, c, k) -> np.ndarray:
        t = np.ascontiguousarray(t, dtype=np.float64)
        c = np.ascontiguousarray(c, dtype=np.complex128)
        k = np.ascontiguousarray(k, dtype=np.int32)
        m, d = t.shape
        K = k.shape[0]
        f = np.zeros(K, dtype=np.complex128)
        _check(self._lib.prony_eval(self._h, _ptr(t), _ptr(c), m, d, _ptr(k), K, _ptr(f)), "prony_eval")
        return f

    def solve_batched(self, grids, ds, ns, ms, opts: PronyOpts | None = None):
        P = len(grids)
        ds = np.asarray(ds, dtype=np.int32)
        ns = np.asarray(ns, dtype=np.int32)
        ms = np.asarray(ms, dtype=np.int32)
        sizes = np.array([(2 * int(n) + 2) ** int(d) for d, n in zip(ds, ns)], dtype=np.int64)
        soff = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        ooff = np.concatenate([[0], np.cumsum(ms)[:-1]]).astype(np.int64)
        samples = np.concatenate([np.ascontiguousarray(g, dtype=np.complex128).reshape(-1) for g in grids])
        total = int(ms.sum())
        dmax = int(ds.max())
        t = np.zeros(total * dmax)
        c = np.zeros(total, dtype=np.complex128)
        infos = (PronyInfo * P)()
        rc = self._lib.prony_solve_batched(self._h, P, _ptr(ds), _ptr(ns), _ptr(ms), _ptr(soff), _ptr(samples),
                                           _ptr(ooff), _ptr(t), _ptr(c), infos,
                                           ctypes.byref(opts) if opts else None)
        if rc in (PRONY_EINVAL, PRONY_ECUDA, PRONY_ENOMEM):
            raise PronyError(rc, "prony_solve_batched")
        out = []
        for i in range(P):
            d, m, o = int(ds[i]), int(ms[i]), int(ooff[i])
            out.append(SolveResult(t[o * dmax:(o + m) * dmax].reshape(m, dmax)[:, :d].copy(), c[o:o + m].copy(),
                                   infos[i].as_dict()))
        return out, rc

    # ---------------------------------------------------------------- device-pointer calls (torch tensors)
    def solve_batched_host(self, samples, ds, ns, ms, soff, ooff, t_out, c_out, opts: PronyOpts | None = None):
        """prony_solve_batched on caller-owned host buffers (numpy arrays or CPU torch tensors, pinned
        or not): packed complex128 samples at soff, t_out (float64) and c_out (complex128) at ooff
        (t rows of the call's largest d).  Returns (infos, worst status)."""
        def ptr(a):
            return ctypes.c_void_p(a.data_ptr()) if hasattr(a, "data_ptr") else _ptr(a)
        P = len(ds)
        ds = np.asarray(ds, dtype=np.int32)
        ns = np.asarray(ns, dtype=np.int32)
        ms = np.asarray(ms, dtype=np.int32)
        soff = np.asarray(soff, dtype=np.int64)
        ooff = np.asarray(ooff, dtype=np.int64)
        infos = (PronyInfo * P)()
        rc = self._lib.prony_solve_batched(self._h, P, _ptr(ds), _ptr(ns), _ptr(ms), _ptr(soff), ptr(samples),
                                           _ptr(ooff), ptr(t_out), ptr(c_out), infos,
                                           ctypes.byref(opts) if opts else None)
        if rc in (PRONY_EINVAL, PRONY_ECUDA, PRONY_ENOMEM):
            raise PronyError(rc, "prony_solve_batched")
        return [i.as_dict() for i in infos], rc

    def solve_batched_dev(self, samples_dev, ds, ns, ms, soff, ooff, t_out_dev, c_out_dev,
                          opts: PronyOpts | None = None, stream: int = 0):
        ds = np.asarray(ds, dtype=np.int32)
        ns = np.asarray(ns, dtype=np.int32)
        ms = np.asarray(ms, dtype=np.int32)
        soff = np.asarray(soff, dtype=np.int64)
        ooff = np.asarray(ooff, dtype=np.int64)
        P = len(ds)
        infos = (PronyInfo * P)()
        rc = self._lib.prony_solve_batched_dev(self._h, P, _ptr(ds), _ptr(ns), _ptr(ms), _ptr(soff),
                                               ctypes.c_void_p(samples_dev.data_ptr()), _ptr(ooff),
                                               ctypes.c_void_p(t_out_dev.data_ptr()),
                                               ctypes.c_void_p(c_out_dev.data_ptr()), infos,
                                               ctypes.byref(opts) if opts else None, ctypes.c_void_p(stream))
        if rc in (PRONY_EINVAL, PRONY_ECUDA, PRONY_ENOMEM):
            raise PronyError(rc, "prony_solve_batched_dev")
        return [infos[i].as_dict() for i in range(P)], rc

    def expsum_fwd_dev(self, t_dev, c_dev, lo, length, f_dev, stream: int = 0):
        m, d = t_dev.shape
        lo = np.ascontiguousarray(lo, dtype=np.int32)
        ln = np.ascontiguousarray(length, dtype=np.int32)
        _check(self._lib.prony_expsum_fwd_dev(self._h, ctypes.c_void_p(t_dev.data_ptr()),
                                              ctypes.c_void_p(c_dev.data_ptr()), m, d, _ptr(lo), _ptr(ln),
                                              ctypes.c_void_p(f_dev.data_ptr()), ctypes.c_void_p(stream)),
               "prony_expsum_fwd_dev")

    def expsum_bwd_dev(self, t_dev, c_dev, lo, length, g_dev, gt_dev, gc_dev, stream: int = 0):
        m, d = t_dev.shape
        lo = np.ascontiguousarray(lo, dtype=np.int32)
        ln = np.ascontiguousarray(length, dtype=np.int32)
        _check(self._lib.prony_expsum_bwd_dev(self._h, ctypes.c_void_p(t_dev.data_ptr()),
                                              ctypes.c_void_p(c_dev.data_ptr()), m, d, _ptr(lo), _ptr(ln),
                                              ctypes.c_void_p(g_dev.data_ptr()), ctypes.c_void_p(gt_dev.data_ptr()),
                                              ctypes.c_void_p(gc_dev.data_ptr()), ctypes.c_void_p(stream)),
               "prony_expsum_bwd_dev")

    def refine_lm_dev(self, t_dev, c_dev, lo, length, y_dev, iters: int, lambda0: float = 1e-3, loss_dev=None,
                      stream: int = 0):
        """Levenberg-Marquardt refinement in place: t_dev (m, d) float64, c_dev (m,) complex128,
        y_dev complex64 samples on the box; loss_dev (iters + 1,) float64 or None."""
        m, d = t_dev.shape
        lo = np.ascontiguousarray(lo, dtype=np.int32)
        ln = np.ascontiguousarray(length, dtype=np.int32)
        _check(self._lib.prony_refine_lm_dev(self._h, ctypes.c_void_p(t_dev.data_ptr()),
                                             ctypes.c_void_p(c_dev.data_ptr()), m, d, _ptr(lo), _ptr(ln),
                                             ctypes.c_void_p(y_dev.data_ptr()), int(iters), float(lambda0),
                                             ctypes.c_void_p(loss_dev.data_ptr() if loss_dev is not None else 0),
                                             ctypes.c_void_p(stream)),
               "prony_refine_lm_dev")

    def toeplitz_mm_dev(self, grid_dev, d: int, n: int, X_dev, L: int, adjoint: int, precision, Y_dev,
                        stream: int = 0):
        r = X_dev.shape[0] if X_dev.dim() == 2 else 1
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        _check(self._lib.prony_toeplitz_mm_dev(self._h, ctypes.c_void_p(grid_dev.data_ptr()), d, n,
                                               ctypes.c_void_p(X_dev.data_ptr()), r, L, adjoint, precision,
                                               ctypes.c_void_p(Y_dev.data_ptr()), ctypes.c_void_p(stream)),
               "prony_toeplitz_mm_dev")
