"""Thin ctypes binding of libkfac (include/kfac.h).

Argument marshalling only: every step of the hot path runs in the CUDA library.
PyTorch supplies device memory and streams. The functions carry the C names and
take CUDA float32 tensors whose rows are contiguous (stride(1) == 1); the row
stride becomes the C leading dimension. There is no CPU fallback: without the
compiled library every call raises.
"""
from __future__ import annotations

import ctypes
import os

# The forked streams of a grouped call run concurrently only as far as the
# CUDA runtime has hardware work queues for them: CUDA_DEVICE_MAX_CONNECTIONS,
# 8 by default, beyond which streams share a queue and one stream's pending
# chain blocks the next. Raise it to the maximum (32) unless the caller chose a
# value; it is read when the process creates its CUDA context, so it takes
# effect when this module is imported before any CUDA work.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import torch  # noqa: E402

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libkfac.so")
_lib = None

PRECISION = {"fp32": 0, "tf32": 1, "bf16": 2}
OPTIONS = {"cholqr_passes": 0, "cholqr_shift": 1, "eig_refine": 2, "eig_max_sweeps": 3, "eig_tol": 4,
           "cholqr_inner_passes": 5, "cholqr_fp32_passes": 6,
           "basis_polish": 7, "cholqr_inner_fp32": 8, "eig_stop_tol": 9, "eig_refine_fp64": 10, "wait_cycles": 11,
           "group_streams": 12, "invert_method": 13,
           "chol_cluster": 14, "split_target": 15, "warm_start": 16,
           "conv_chunk": 17, "chol_panel": 18, "tail_planes": 19,
           "chol_blocked": 20, "trsm_inverse": 21}
FLAGS = {1: "CHOL_SHIFTED", 2: "CHOL_FAILED", 4: "EIG_NOCONV", 8: "NONFINITE", 16: "EIG_SHIFTED", 32: "TIMEOUT"}


class KfacError(RuntimeError):
    pass


class InvertDesc(ctypes.Structure):
    """Mirror of kfac_invert_desc."""
    _fields_ = [("d", ctypes.c_int), ("F", ctypes.c_void_p), ("ldf", ctypes.c_int), ("rank", ctypes.c_int),
                ("oversample", ctypes.c_int), ("power_iters", ctypes.c_int), ("lam", ctypes.c_float),
                ("omega", ctypes.c_void_p), ("ldo", ctypes.c_int), ("prec", ctypes.c_int), ("U", ctypes.c_void_p),
                ("ldu", ctypes.c_int), ("D", ctypes.c_void_p), ("coef", ctypes.c_void_p), ("seed", ctypes.c_uint64)]


class EaDesc(ctypes.Structure):
    """Mirror of kfac_ea_desc."""
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.c_int), ("X", ctypes.c_void_p), ("ldx", ctypes.c_int),
                ("rho", ctypes.c_float), ("prec", ctypes.c_int), ("F", ctypes.c_void_p), ("ldf", ctypes.c_int)]


class PrecondDesc(ctypes.Structure):
    """Mirror of kfac_precond_desc."""
    _fields_ = [("d_g", ctypes.c_int), ("d_a", ctypes.c_int), ("J", ctypes.c_void_p), ("ldj", ctypes.c_int),
                ("U_a", ctypes.c_void_p), ("ld_ua", ctypes.c_int), ("coef_a", ctypes.c_void_p), ("r_a", ctypes.c_int),
                ("U_g", ctypes.c_void_p), ("ld_ug", ctypes.c_int), ("coef_g", ctypes.c_void_p), ("r_g", ctypes.c_int),
                ("lam", ctypes.c_float), ("prec", ctypes.c_int), ("S", ctypes.c_void_p), ("lds", ctypes.c_int)]


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libkfac.so (built in-tree by build.py); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise KfacError(f"{_LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(_LIB_PATH)
        vp, i, f, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double, ctypes.c_int64
        L.kfac_version.restype = i
        L.kfac_status_string.argtypes = [i]
        L.kfac_status_string.restype = ctypes.c_char_p
        L.kfac_create.argtypes = [ctypes.POINTER(vp), i, vp]
        L.kfac_destroy.argtypes = [vp]
        L.kfac_set_stream.argtypes = [vp, vp]
        L.kfac_reserve.argtypes = [vp, i, i, i64]
        L.kfac_set_option.argtypes = [vp, i, d]
        L.kfac_get_status.argtypes = [vp, ctypes.POINTER(i)]
        L.kfac_ea_update_conv.argtypes = [vp, i, i, i, i, vp, i, i, i, i, i, i, i, f, f, i, vp, i]
        L.kfac_ea_update_conv.restype = i
        L.kfac_ea_update_rows.argtypes = [vp, i, i, vp, i, i, f, f, i, vp, i]
        L.kfac_ea_update_rows.restype = i
        L.kfac_autotune_invert.argtypes = [vp, i, ctypes.POINTER(InvertDesc), ctypes.c_char_p, ctypes.POINTER(i)]
        L.kfac_autotune_invert.restype = i
        L.kfac_get_item_status.argtypes = [vp, i, ctypes.POINTER(i)]
        L.kfac_get_item_status.restype = i
        L.kfac_ea_update.argtypes = [vp, i, i, vp, i, f, i, vp, i]
        L.kfac_rsvd_invert.argtypes = [vp, i, vp, i, i, i, i, f, vp, i, ctypes.c_uint64, i, vp, i, vp, vp]
        L.kfac_draw_omega.argtypes = [vp, i, i, ctypes.c_uint64, vp, i]
        L.kfac_precondition.argtypes = [vp, i, i, vp, i, vp, i, vp, i, vp, i, vp, i, f, i, vp, i]
        L.kfac_profile_enable.argtypes = [vp, i]
        L.kfac_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(d), ctypes.POINTER(i), i,
                                        ctypes.POINTER(i)]
        L.kfac_profile_timeline.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(d),
                                            ctypes.POINTER(d), ctypes.POINTER(i)]
        L.kfac_profile_timeline.restype = i
        L.kfac_stage_name.argtypes = [i]
        L.kfac_stage_name.restype = ctypes.c_char_p
        L.kfac_kernel_launch_count.restype = ctypes.c_uint64
        L.kfac_simt_gemm_count.restype = ctypes.c_uint64
        L.kfac_rsvd_invert_grouped.argtypes = [vp, i, ctypes.POINTER(InvertDesc)]
        L.kfac_ea_update_grouped.argtypes = [vp, i, ctypes.POINTER(EaDesc)]
        L.kfac_ea_update_grouped.restype = i
        L.kfac_precondition_grouped.argtypes = [vp, i, ctypes.POINTER(PrecondDesc)]
        L.kfac_precondition_grouped.restype = i
        L.kfac_step_grouped.argtypes = [vp, i, ctypes.POINTER(EaDesc), ctypes.POINTER(InvertDesc), i,
                                        ctypes.POINTER(PrecondDesc), ctypes.POINTER(i)]
        L.kfac_step_grouped.restype = i
        L.kfac_gemm_nt.argtypes = [vp, i, i, i, vp, i, vp, i, f, f, vp, i, i]
        L.kfac_gemm_nt.restype = i
        L.kfac_rsvd_invert_grouped.restype = i
        L.kfac_precondition_noalloc.argtypes = [vp, i, i, vp, i, vp, i, vp, i, vp, i, vp, i, f, i, vp, i]
        L.kfac_precondition_noalloc.restype = i
        L.kfac_stats_read.argtypes = [vp, ctypes.POINTER(i64), i]
        for name in ("kfac_create", "kfac_destroy", "kfac_set_stream", "kfac_reserve", "kfac_set_option",
                     "kfac_get_status", "kfac_ea_update", "kfac_rsvd_invert", "kfac_precondition",
                     "kfac_profile_enable", "kfac_profile_read", "kfac_stats_read"):
            getattr(L, name).restype = i
        _lib = L
    return _lib


def _check(st: int, what: str):
    if st != 0:
        raise KfacError(f"{what}: {lib().kfac_status_string(st).decode()}")


def _mat(t: torch.Tensor, name: str, rows: int | None = None, cols: int | None = None):
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.float32 or t.dim() != 2:
        raise KfacError(f"{name} must be a 2-D CUDA float32 tensor")
    if t.shape[1] > 1 and t.stride(1) != 1:
        raise KfacError(f"{name} rows must be contiguous")
    if (rows is not None and t.shape[0] != rows) or (cols is not None and t.shape[1] != cols):
        raise KfacError(f"{name} has shape {tuple(t.shape)}, expected ({rows}, {cols})")
    return ctypes.c_void_p(t.data_ptr()), max(t.stride(0), t.shape[1], 1)


def _vec(t: torch.Tensor, name: str, n: int):
    if t.device.type != "cuda" or t.dtype != torch.float32 or t.dim() != 1 or t.shape[0] != n or (n > 1 and t.stride(0) != 1):
        raise KfacError(f"{name} must be a contiguous CUDA float32 vector of length {n}")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """Owns a kfac_ctx (workspace + status word) bound to one device and stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.device = torch.device("cuda", device)
        torch.cuda.init()
        self._stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _check(lib().kfac_create(ctypes.byref(h), device, ctypes.c_void_p(self._stream.cuda_stream)), "kfac_create")
        self.handle = h

    @property
    def stream(self) -> torch.cuda.Stream:
        return self._stream

    def set_stream(self, stream: torch.cuda.Stream):
        _check(lib().kfac_set_stream(self.handle, ctypes.c_void_p(stream.cuda_stream)), "kfac_set_stream")
        self._stream = stream

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().kfac_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def kfac_set_option(ctx: Context, name: str, value: float):
    _check(lib().kfac_set_option(ctx.handle, OPTIONS[name], float(value)), f"kfac_set_option({name})")


def kfac_reserve(ctx: Context, d_max: int, k_max: int, mn_max: int = 0):
    _check(lib().kfac_reserve(ctx.handle, int(d_max), int(k_max), int(mn_max)), "kfac_reserve")


def kfac_get_status(ctx: Context):
    """Synchronise the context stream; return (status code, list of raised flag names)."""
    f = ctypes.c_int(0)
    st = lib().kfac_get_status(ctx.handle, ctypes.byref(f))
    return st, [n for b, n in FLAGS.items() if f.value & b]


def kfac_autotune_invert(ctx: Context, descs, cache_path: str | None = None) -> dict:
    """Tune the grouped inversion's schedule for a prepared descriptor array
    (invert_descs); returns the chosen settings."""
    out = (ctypes.c_int * 7)()
    _check(lib().kfac_autotune_invert(ctx.handle, len(descs), descs,
                                      cache_path.encode() if cache_path else None, out), "kfac_autotune_invert")
    return {"group_streams": out[0], "chol_cluster": out[1], "split_target": out[2], "chol_panel": out[3],
            "chol_blocked": out[4], "trsm_inverse": out[5], "cached": bool(out[6])}


def kfac_get_item_status(ctx: Context, count: int):
    """Per-item flag names of grouped calls since the last kfac_get_status (does not clear)."""
    arr = (ctypes.c_int * max(count, 1))()
    _check(lib().kfac_get_item_status(ctx.handle, int(count), arr), "kfac_get_item_status")
    return [[n for b, n in FLAGS.items() if arr[i] & b] for i in range(count)]


def kfac_ea_update(ctx: Context, X: torch.Tensor, F: torch.Tensor, rho: float, prec: str = "fp32"):
    """F <- rho F + (1 - rho)/n X X^T in place; X is (d, n)."""
    d, n = X.shape
    px, ldx = _mat(X, "X", d, n)
    pf, ldf = _mat(F, "F", d, d)
    _check(lib().kfac_ea_update(ctx.handle, d, n, px, ldx, float(rho), PRECISION[prec], pf, ldf), "kfac_ea_update")
    return F


def kfac_ea_update_rows(ctx: Context, A: torch.Tensor, F: torch.Tensor, rho: float, append_one: bool = False,
                        scale: float = 1.0, prec: str = "fp32"):
    """F <- rho F + (1 - rho)/n scale^2 [A, 1]^T [A, 1] in place for a batch A of shape (n, cols)."""
    n, cols = A.shape
    d = cols + int(bool(append_one))
    pa, lda = _mat(A, "A", n, cols)
    pf, ldf = _mat(F, "F", d, d)
    _check(lib().kfac_ea_update_rows(ctx.handle, n, cols, pa, lda, int(bool(append_one)), float(scale), float(rho),
                                     PRECISION[prec], pf, ldf), "kfac_ea_update_rows")
    return F


def kfac_ea_update_conv(ctx: Context, x: torch.Tensor, F: torch.Tensor, kernel, rho: float, stride=(1, 1),
                        padding=(0, 0), append_one: bool = False, scale: float = 1.0, prec: str = "fp32"):
    """Conv-layer factor from the patch statistics of x (n, c, h, w), updated in place."""
    if (not isinstance(x, torch.Tensor) or x.device.type != "cuda" or x.dtype != torch.float32 or x.dim() != 4
            or not x.is_contiguous()):
        raise KfacError("x must be a contiguous 4-D CUDA float32 tensor (NCHW)")
    n, c, h, w = x.shape
    kh, kw = kernel
    d = c * kh * kw + int(bool(append_one))
    pf, ldf = _mat(F, "F", d, d)
    _check(lib().kfac_ea_update_conv(ctx.handle, n, c, h, w, ctypes.c_void_p(x.data_ptr()), kh, kw, stride[0],
                                     stride[1], padding[0], padding[1], int(bool(append_one)), float(scale),
                                     float(rho), PRECISION[prec], pf, ldf), "kfac_ea_update_conv")
    return F


def kfac_rsvd_invert(ctx: Context, F: torch.Tensor, rank: int, oversample: int, power_iters: int, lam: float,
                     omega: torch.Tensor | None, prec: str = "fp32", out=None, seed: int = 0):
    """Randomized low-rank eigendecomposition of F and the damping coefficients.
    Returns (U (d x r), D (r), coef (r)) with r = min(rank, d). omega None: the
    library draws the test matrix of `seed` on the device (kfac_draw_omega)."""
    d = F.shape[0]
    r = min(rank, d)
    pf, ldf = _mat(F, "F", d, d)
    k = rank + oversample
    if omega is not None:
        po, ldo = _mat(omega, "omega", d, k)
    else:
        po, ldo = ctypes.c_void_p(0), max(k, 1)
    if out is None:
        U = torch.empty((d, r), device=F.device, dtype=torch.float32)
        D = torch.empty((r,), device=F.device, dtype=torch.float32)
        coef = torch.empty((r,), device=F.device, dtype=torch.float32)
    else:
        U, D, coef = out
    pu, ldu = _mat(U, "U", d, r)
    _check(lib().kfac_rsvd_invert(ctx.handle, d, pf, ldf, int(rank), int(oversample), int(power_iters), float(lam),
                                  po, ldo, int(seed) & 0xFFFFFFFFFFFFFFFF, PRECISION[prec], pu, ldu,
                                  _vec(D, "D", r), _vec(coef, "coef", r)),
           "kfac_rsvd_invert")
    return U, D, coef


def kfac_draw_omega(ctx: Context, d: int, k: int, seed: int, out: torch.Tensor | None = None) -> torch.Tensor:
    """The library's seeded Gaussian test matrix (d x k), drawn on the device."""
    om = torch.empty((d, k), device=ctx.device, dtype=torch.float32) if out is None else out
    po, ldo = _mat(om, "omega", d, k)
    _check(lib().kfac_draw_omega(ctx.handle, int(d), int(k), int(seed) & 0xFFFFFFFFFFFFFFFF, po, ldo),
           "kfac_draw_omega")
    return om


def kfac_precondition(ctx: Context, J: torch.Tensor, U_a: torch.Tensor, coef_a: torch.Tensor, U_g: torch.Tensor,
                      coef_g: torch.Tensor, lam: float, prec: str = "fp32", out: torch.Tensor | None = None):
    """S = (U_g D_g U_g^T + lam I)^-1 J (U_a D_a U_a^T + lam I)^-1 through Eq. (13) coefficients."""
    dg, da = J.shape
    ra, rg = U_a.shape[1], U_g.shape[1]
    pj, ldj = _mat(J, "J", dg, da)
    pua, ldua = _mat(U_a, "U_a", da, ra)
    pug, ldug = _mat(U_g, "U_g", dg, rg)
    S = torch.empty_like(J) if out is None else out
    ps, lds = _mat(S, "S", dg, da)
    _check(lib().kfac_precondition(ctx.handle, dg, da, pj, ldj, pua, ldua, _vec(coef_a, "coef_a", ra), ra,
                                   pug, ldug, _vec(coef_g, "coef_g", rg), rg, float(lam), PRECISION[prec], ps, lds),
           "kfac_precondition")
    return S


def kfac_profile_enable(ctx: Context, on: bool = True):
    _check(lib().kfac_profile_enable(ctx.handle, int(bool(on))), "kfac_profile_enable")


def kfac_profile_read(ctx: Context) -> dict:
    """{stage name: (device ms summed over timed launches, launch count)}; clears the totals."""
    n = 32
    names = (ctypes.c_char_p * n)()
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int * n)()
    got = ctypes.c_int(0)
    _check(lib().kfac_profile_read(ctx.handle, names, ms, cnt, n, ctypes.byref(got)), "kfac_profile_read")
    return {names[i].decode(): (ms[i], cnt[i]) for i in range(got.value)}


def kfac_profile_timeline(ctx: Context) -> list:
    """Recorded stage intervals [(stage name, item or -1, start ms, end ms)] in
    order of start (call before kfac_profile_read, which clears them)."""
    total = ctypes.c_int(0)
    _check(lib().kfac_profile_timeline(ctx.handle, 0, None, None, None, None, ctypes.byref(total)),
           "kfac_profile_timeline")
    n = total.value
    st, it = (ctypes.c_int * max(n, 1))(), (ctypes.c_int * max(n, 1))()
    a, b = (ctypes.c_double * max(n, 1))(), (ctypes.c_double * max(n, 1))()
    _check(lib().kfac_profile_timeline(ctx.handle, n, st, it, a, b, ctypes.byref(total)), "kfac_profile_timeline")
    return [(lib().kfac_stage_name(st[e]).decode(), it[e], a[e], b[e]) for e in range(min(n, total.value))]


def kfac_kernel_launch_count() -> int:
    return int(lib().kfac_kernel_launch_count())


def kfac_simt_gemm_count() -> int:
    """Large products that ran on the SIMT fallback instead of the tensor cores (process total)."""
    return int(lib().kfac_simt_gemm_count())


def kfac_stats_read(ctx: Context) -> dict:
    out = (ctypes.c_int64 * 4)()
    _check(lib().kfac_stats_read(ctx.handle, out, 4), "kfac_stats_read")
    return {"jacobi_sweeps": out[0], "jacobi_solves": out[1], "cholesky": out[2], "cholesky_retries": out[3]}


NOALLOC_SCRATCH_FLOATS = 2 * 1024 * 1024


def kfac_precondition_noalloc(J: torch.Tensor, U_a: torch.Tensor, coef_a: torch.Tensor, U_g: torch.Tensor,
                              coef_g: torch.Tensor, lam: float, prec: str = "fp32", out: torch.Tensor | None = None,
                              stream: torch.cuda.Stream | None = None):
    """kfac_precondition without any device allocation inside the library: for
    callers that cannot allocate at call time (graph capture, pre-reserved memory
    pools). Runs on `stream` (default: the current stream) of J's device; the
    output tensor must be supplied by the caller or is allocated here by torch."""
    dg, da = J.shape
    ra, rg = U_a.shape[1], U_g.shape[1]
    pj, ldj = _mat(J, "J", dg, da)
    pua, ldua = _mat(U_a, "U_a", da, ra)
    pug, ldug = _mat(U_g, "U_g", dg, rg)
    S = torch.empty_like(J) if out is None else out
    ps, lds = _mat(S, "S", dg, da)
    st = stream if stream is not None else torch.cuda.current_stream(J.device)
    with torch.cuda.device(J.device):
        _check(lib().kfac_precondition_noalloc(ctypes.c_void_p(st.cuda_stream), dg, da, pj, ldj, pua, ldua,
                                               _vec(coef_a, "coef_a", ra), ra, pug, ldug,
                                               _vec(coef_g, "coef_g", rg), rg, float(lam), PRECISION[prec], ps, lds),
               "kfac_precondition_noalloc")
    return S


def invert_descs(items):
    """kfac_invert_desc array for a grouped inversion. items: sequence of dicts
    with keys F, rank, oversample, power_iters, lam, omega (None: drawn from the
    key seed on the device), prec (optional) and out (optional (U, D, coef)). Returns (descs, [(U, D, coef), ...]); the array
    can be passed to call_grouped() any number of times."""
    descs = (InvertDesc * len(items))()
    outs = []
    for it, dsc in zip(items, descs):
        F = it["F"]
        d = F.shape[0]
        r = min(it["rank"], d)
        k = it["rank"] + it["oversample"]
        pf, ldf = _mat(F, "F", d, d)
        om = it.get("omega")
        po, ldo = _mat(om, "omega", d, k) if om is not None else (ctypes.c_void_p(0), max(k, 1))
        if it.get("out") is None:
            U = torch.empty((d, r), device=F.device, dtype=torch.float32)
            D = torch.empty((r,), device=F.device, dtype=torch.float32)
            coef = torch.empty((r,), device=F.device, dtype=torch.float32)
        else:
            U, D, coef = it["out"]
        pu, ldu = _mat(U, "U", d, r)
        dsc.d, dsc.F, dsc.ldf = d, pf.value, ldf
        dsc.rank, dsc.oversample, dsc.power_iters = int(it["rank"]), int(it["oversample"]), int(it["power_iters"])
        dsc.lam, dsc.omega, dsc.ldo = float(it["lam"]), po.value, ldo
        dsc.seed = int(it.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
        dsc.prec = PRECISION[it.get("prec", "fp32")]
        dsc.U, dsc.ldu = pu.value, ldu
        dsc.D, dsc.coef = _vec(D, "D", r).value, _vec(coef, "coef", r).value
        outs.append((U, D, coef))
    return descs, outs


def ea_descs(items):
    """kfac_ea_desc array for a grouped EA update. items: sequence of dicts with
    keys X (d x n), F (d x d, updated in place), rho and prec (optional)."""
    descs = (EaDesc * len(items))()
    for it, dsc in zip(items, descs):
        F, X = it["F"], it["X"]
        d, n = X.shape
        px, ldx = _mat(X, "X", d, n)
        pf, ldf = _mat(F, "F", d, d)
        dsc.d, dsc.n, dsc.X, dsc.ldx = d, n, px.value, ldx
        dsc.rho, dsc.prec, dsc.F, dsc.ldf = float(it["rho"]), PRECISION[it.get("prec", "fp32")], pf.value, ldf
    return descs


def precond_descs(items):
    """kfac_precond_desc array for a grouped apply. items: sequence of dicts with
    keys J, U_a, coef_a, U_g, coef_g, lam, prec (optional) and out (optional S).
    Returns (descs, [S, ...])."""
    descs = (PrecondDesc * len(items))()
    outs = []
    for it, dsc in zip(items, descs):
        J, Ua, Ug = it["J"], it["U_a"], it["U_g"]
        dg, da = J.shape
        ra, rg = Ua.shape[1], Ug.shape[1]
        pj, ldj = _mat(J, "J", dg, da)
        pua, ldua = _mat(Ua, "U_a", da, ra)
        pug, ldug = _mat(Ug, "U_g", dg, rg)
        S = torch.empty_like(J) if it.get("out") is None else it["out"]
        ps, lds = _mat(S, "S", dg, da)
        dsc.d_g, dsc.d_a, dsc.J, dsc.ldj = dg, da, pj.value, ldj
        dsc.U_a, dsc.ld_ua, dsc.coef_a, dsc.r_a = pua.value, ldua, _vec(it["coef_a"], "coef_a", ra).value, ra
        dsc.U_g, dsc.ld_ug, dsc.coef_g, dsc.r_g = pug.value, ldug, _vec(it["coef_g"], "coef_g", rg).value, rg
        dsc.lam, dsc.prec, dsc.S, dsc.lds = float(it["lam"]), PRECISION[it.get("prec", "fp32")], ps.value, lds
        outs.append(S)
    return descs, outs


_GROUPED = {"ea": "kfac_ea_update_grouped", "invert": "kfac_rsvd_invert_grouped",
            "precondition": "kfac_precondition_grouped"}


def step_descs(layer_factors):
    """int array of (A factor, G factor) per layer for kfac_step_grouped (-1: none)."""
    flat = [int(v) for pair in layer_factors for v in pair]
    return (ctypes.c_int * max(len(flat), 1))(*flat)


def kfac_step_grouped(ctx: Context, ea, inv, pre, layer_factors):
    """One step on prepared descriptor arrays (ea_descs or None, invert_descs,
    precond_descs) and a step_descs array of each layer's two factor indices."""
    n_l = len(pre)
    _check(lib().kfac_step_grouped(ctx.handle, len(inv), ea, inv, n_l, pre, layer_factors), "kfac_step_grouped")


def call_grouped(ctx: Context, kind: str, descs):
    """Issue a grouped call ("ea", "invert" or "precondition") on a prepared descriptor array."""
    name = _GROUPED[kind]
    _check(getattr(lib(), name)(ctx.handle, len(descs), descs), name)


def kfac_rsvd_invert_grouped(ctx: Context, items):
    """Grouped kfac_rsvd_invert (items as invert_descs). Returns the list of (U, D, coef)."""
    descs, outs = invert_descs(items)
    call_grouped(ctx, "invert", descs)
    return outs


def kfac_ea_update_grouped(ctx: Context, items):
    """Grouped kfac_ea_update (items as ea_descs)."""
    call_grouped(ctx, "ea", ea_descs(items))
    return [it["F"] for it in items]


def kfac_precondition_grouped(ctx: Context, items):
    """Grouped kfac_precondition (items as precond_descs). Returns the list of S."""
    descs, outs = precond_descs(items)
    call_grouped(ctx, "precondition", descs)
    return outs


def kfac_gemm_nt(ctx: Context, A: torch.Tensor, B: torch.Tensor, D: torch.Tensor, alpha: float = 1.0,
                 beta: float = 0.0, prec: str = "fp32"):
    """D = alpha A B^T + beta D (GEMM engine utility)."""
    M, K = A.shape
    N = B.shape[0]
    pa, lda = _mat(A, "A", M, K)
    pb, ldb = _mat(B, "B", N, K)
    pd, ldd = _mat(D, "D", M, N)
    _check(lib().kfac_gemm_nt(ctx.handle, M, N, K, pa, lda, pb, ldb, float(alpha), float(beta), pd, ldd,
                              PRECISION[prec]), "kfac_gemm_nt")
    return D
