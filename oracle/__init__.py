"""FP64 CPU oracle for the randomized K-FAC hot path (Puiu, arXiv 2206.15397).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The CUDA library never
imports, links or executes anything here, and this package shares no code with
it (the only common dependency is the seeded input generator, which holds none
of the method's arithmetic).

The arithmetic lives in ``oracle.c`` (plain sequential FP64 C); this module
compiles it with gcc on first use and wraps it with ctypes. Every wrapper takes
and returns float64 numpy arrays, row-major.

Functions and the passages they follow:
  ea_update        Alg. 1, EA update of the forward/backward K-factors; Eq. (6)
  ea_update_conv   the same for a conv layer, from patch statistics (Sec. 2.1's conv K-factors)
  jacobi_eigh      "eig" of Alg. 1 / "Eigen_decomp" of Alg. 3 (cyclic Jacobi)
  qr               "QR_decomp" of Alg. 2 / Alg. 3 (Householder)
  srevd            Alg. 3 with the power iteration of Sec. 2.2
  svd_jacobi       the "full SVD" of Alg. 2 (one-sided Hestenes Jacobi)
  rsvd             Alg. 2 with the power iteration of Sec. 2.2, returning V~ (RS-KFAC, Alg. 4)
  damped_coef      Eq. (13), the diagonal (D + lam I)^-1 - I/lam
  precondition     Alg. 4, the M and S updates (Alg. 5 supplies U~ for V~)
  precondition_cols  the same S, selected columns only (full-size sampled checks)
  exact_apply      Alg. 1, eig + M/S updates: (G + lam I)^-1 J (A + lam I)^-1
  rank_bound       Proposition 3.1, Eq. (7)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (plain gcc, -O2, no arch flags;
    -fopenmp spreads independent rows over the host cores without changing any
    sum's order; OMP_NUM_THREADS caps the threads)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int) -> int:
    """Set the OpenMP thread count of later oracle calls; returns the previous maximum."""
    lib = _load()
    prev = lib.omp_get_max_threads()
    lib.omp_set_num_threads(int(n))
    return prev


def max_threads() -> int:
    return int(_load().omp_get_max_threads())


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i, d, l = ctypes.c_int, ctypes.c_double, ctypes.c_long
            lib.orc_matmul.argtypes = [i, i, i, _dp, i, _dp, i, _dp]
            lib.orc_ea_update.argtypes = [i, i, _dp, d, _dp]
            lib.orc_jacobi_eigh.argtypes = [i, _dp, _dp, _dp, i, d]
            lib.orc_jacobi_eigh.restype = i
            lib.orc_qr.argtypes = [i, i, _dp, _dp, _dp]
            lib.orc_srevd.argtypes = [i, _dp, i, _dp, i, i, _dp, _dp, _dp, _dp]
            lib.orc_srevd.restype = i
            lib.orc_damped_coef.argtypes = [i, _dp, d, _dp]
            lib.orc_ea_update_conv.argtypes = [i, i, i, i, _dp, i, i, i, i, i, i, i, d, d, _dp]
            lib.orc_svd_jacobi.argtypes = [i, i, _dp, _dp, _dp, _dp, i, d]
            lib.orc_svd_jacobi.restype = i
            lib.orc_rsvd.argtypes = [i, _dp, i, _dp, i, i, _dp, _dp, _dp]
            lib.orc_rsvd.restype = i
            lib.orc_precondition.argtypes = [i, i, _dp, _dp, _dp, i, _dp, _dp, i, d, _dp]
            ip = ctypes.POINTER(ctypes.c_int)
            lib.orc_precondition_cols.argtypes = [i, i, _dp, _dp, _dp, i, _dp, _dp, i, d, i, ip, _dp]
            lib.orc_exact_apply.argtypes = [i, i, _dp, _dp, _dp, d, _dp]
            lib.orc_exact_apply.restype = i
            lib.orc_rank_bound.argtypes = [d, d, d, l, l]
            lib.orc_rank_bound.restype = l
            lib.omp_get_max_threads.restype = i
            lib.omp_set_num_threads.argtypes = [i]
            _lib = lib
    return _lib


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def matmul(a, b, ta: bool = False, tb: bool = False) -> np.ndarray:
    """op(a) @ op(b) by plain triple loop (used by tests to keep the oracle library-free)."""
    a, b = _c(a), _c(b)
    m, kk = (a.shape[1], a.shape[0]) if ta else a.shape
    n = b.shape[0] if tb else b.shape[1]
    out = np.empty((m, n))
    _load().orc_matmul(m, n, kk, _p(a), int(ta), _p(b), int(tb), _p(out))
    return out


def ea_update(factor, x, rho: float) -> np.ndarray:
    """Return rho * factor + (1 - rho) * x x^T / n for x of shape (d, n)."""
    f = _c(factor).copy()
    x = _c(x)
    d, n = x.shape
    assert f.shape == (d, d)
    _load().orc_ea_update(d, n, _p(x), float(rho), _p(f))
    return f


def ea_update_conv(factor, x, kernel, stride=(1, 1), pad=(0, 0), rho: float = 0.95, append_one: bool = False,
                   scale: float = 1.0) -> np.ndarray:
    """EA update of a conv layer's factor from the patch statistics of x (n, c, h, w)."""
    f = _c(factor).copy()
    x = _c(x)
    n, c, h, w = x.shape
    kh, kw = kernel
    d = c * kh * kw + int(append_one)
    assert f.shape == (d, d)
    _load().orc_ea_update_conv(n, c, h, w, _p(x), kh, kw, stride[0], stride[1], pad[0], pad[1], int(append_one),
                               float(scale), float(rho), _p(f))
    return f


def jacobi_eigh(a, max_sweeps: int = 100, tol: float = 1e-15):
    """Cyclic Jacobi: returns (w descending, V with eigenvectors in columns, sweeps)."""
    a = _c(a)
    n = a.shape[0]
    w = np.empty(n)
    v = np.empty((n, n))
    sweeps = _load().orc_jacobi_eigh(n, _p(a), _p(w), _p(v), int(max_sweeps), float(tol))
    return w, v, sweeps


def qr(y):
    """Householder thin QR with non-negative diag(R): returns (Q, R)."""
    y = _c(y)
    m, k = y.shape
    assert m >= k
    q = np.empty((m, k))
    r = np.empty((k, k))
    _load().orc_qr(m, k, _p(y), _p(q), _p(r))
    return q, r


def srevd(factor, omega, power_iters: int, rank: int, return_basis: bool = False):
    """Alg. 3 + power iterations. Returns (U d x r, D r) [, Q, C when return_basis]."""
    f = _c(factor)
    om = _c(omega)
    d = f.shape[0]
    k = om.shape[1]
    r = min(rank, d)
    u = np.empty((d, r))
    dd = np.empty(r)
    qb = np.empty((d, k)) if (return_basis and k < d) else None
    cb = np.empty((k, k)) if (return_basis and k < d) else None
    rc = _load().orc_srevd(d, _p(f), k, _p(om), int(power_iters), int(rank), _p(u), _p(dd),
                           _p(qb) if qb is not None else None, _p(cb) if cb is not None else None)
    if rc < 0:
        raise RuntimeError("oracle Jacobi did not converge")
    if return_basis:
        return u, dd, qb, cb
    return u, dd


def svd_jacobi(a, max_sweeps: int = 100, tol: float = 1e-15):
    """One-sided Jacobi thin SVD of a (m x n, m >= n): returns (U, s descending, V, sweeps)."""
    a = _c(a)
    m, n = a.shape
    assert m >= n
    u = np.empty((m, n))
    s = np.empty(n)
    v = np.empty((n, n))
    sweeps = _load().orc_svd_jacobi(m, n, _p(a), _p(u), _p(s), _p(v), int(max_sweeps), float(tol))
    return u, s, v, sweeps


def rsvd(factor, omega, power_iters: int, rank: int, return_u: bool = False):
    """Alg. 2 + power iterations on a symmetric PSD factor: returns (V~ d x r, S~ r)
    [, U~ d x r when return_u]."""
    f = _c(factor)
    om = _c(omega)
    d = f.shape[0]
    k = om.shape[1]
    r = min(rank, d)
    v = np.empty((d, r))
    s = np.empty(r)
    u = np.empty((d, r)) if return_u else None
    rc = _load().orc_rsvd(d, _p(f), k, _p(om), int(power_iters), int(rank), _p(v), _p(s),
                          _p(u) if u is not None else None)
    if rc < 0:
        raise RuntimeError("oracle Jacobi did not converge")
    return (v, s, u) if return_u else (v, s)


def invert_rsvd(factor, omega, rank: int, power_iters: int, lam: float):
    """The RS-KFAC inversion (Alg. 2 for V~ and S~, Eq. (13) coefficients): (V~, S~, coef)."""
    v, s = rsvd(factor, omega, power_iters, rank)
    return v, s, damped_coef(s, lam)


def damped_coef(dvals, lam: float) -> np.ndarray:
    dv = _c(dvals)
    out = np.empty_like(dv)
    _load().orc_damped_coef(dv.shape[0], _p(dv), float(lam), _p(out))
    return out


def precondition(j, ua, ca, ug, cg, lam: float) -> np.ndarray:
    j, ua, ca, ug, cg = _c(j), _c(ua), _c(ca), _c(ug), _c(cg)
    dg, da = j.shape
    s = np.empty((dg, da))
    _load().orc_precondition(dg, da, _p(j), _p(ua), _p(ca), ua.shape[1], _p(ug), _p(cg), ug.shape[1],
                             float(lam), _p(s))
    return s


def precondition_cols(j, ua, ca, ug, cg, lam: float, cols) -> np.ndarray:
    """Columns `cols` of precondition(j, ua, ca, ug, cg, lam), shape (d_g, len(cols))."""
    j, ua, ca, ug, cg = _c(j), _c(ua), _c(ca), _c(ug), _c(cg)
    dg, da = j.shape
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    assert cols.ndim == 1 and np.all((cols >= 0) & (cols < da))
    out = np.empty((dg, cols.shape[0]))
    _load().orc_precondition_cols(dg, da, _p(j), _p(ua), _p(ca), ua.shape[1], _p(ug), _p(cg), ug.shape[1],
                                  float(lam), int(cols.shape[0]), cols.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  _p(out))
    return out


def exact_apply(j, fa, fg, lam: float) -> np.ndarray:
    j, fa, fg = _c(j), _c(fa), _c(fg)
    dg, da = j.shape
    s = np.empty((dg, da))
    rc = _load().orc_exact_apply(dg, da, _p(j), _p(fa), _p(fg), float(lam), _p(s))
    if rc < 0:
        raise RuntimeError("oracle Jacobi did not converge")
    return s


def rank_bound(eps: float, alpha: float, rho: float, n_m: int, d_m: int) -> int:
    return int(_load().orc_rank_bound(float(eps), float(alpha), float(rho), int(n_m), int(d_m)))


def invert(factor, omega, rank: int, power_iters: int, lam: float):
    """Full randomized inversion as the GPU computes it: (U, D, coef)."""
    u, dd = srevd(factor, omega, power_iters, rank)
    return u, dd, damped_coef(dd, lam)
