"""The allocation-free preconditioner entry point (kfac_precondition_noalloc).

Some callers cannot allocate GPU memory when they call the library (work
recorded during CUDA graph capture, frameworks that reserve all device memory
up front); this entry point keeps its scratch in a static device array. It must
agree with kfac_precondition on the same inputs, call after call, although every
call reuses the same scratch. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle


def _lib():
    from paper_2206_15397_gb300 import build, kfac
    build.build()
    return kfac


def test_noalloc_rejects_oversized_requests_before_any_work():
    kf = _lib()
    L = kf.lib()
    big = kf.NOALLOC_SCRATCH_FLOATS // 100 + 1   # d_g * r_a = 100 * big > the scratch
    dummy = ctypes.c_void_p(16)                  # never dereferenced: the size check comes first
    st = L.kfac_precondition_noalloc(None, big, 200, dummy, 200, dummy, 100, dummy, 100, dummy, 1, dummy, 1,
                                     ctypes.c_float(0.1), 0, ctypes.c_void_p(32), 200)
    assert L.kfac_status_string(st) == b"KFAC_ERR_TOO_LARGE"


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
def test_noalloc_matches_precondition_twice(prec):
    torch = pytest.importorskip("torch")
    kf = _lib()
    dev = torch.device("cuda", 0)
    with kf.Context(0) as ctx:
        for call, (dg, da, rg, ra) in enumerate([(300, 513, 40, 64), (257, 130, 17, 0), (96, 200, 0, 30)]):
            rng = np.random.default_rng(100 + call)
            ua = np.linalg.qr(rng.standard_normal((da, max(ra, 1))))[0][:, :ra].astype(np.float32)
            ug = np.linalg.qr(rng.standard_normal((dg, max(rg, 1))))[0][:, :rg].astype(np.float32)
            lam = 0.1
            ca = oracle.damped_coef(np.sort(rng.uniform(0, 3, ra))[::-1], lam).astype(np.float32)
            cg = oracle.damped_coef(np.sort(rng.uniform(0, 3, rg))[::-1], lam).astype(np.float32)
            j = rng.standard_normal((dg, da)).astype(np.float32)
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
            J, Ua, Ca, Ug, Cg = t(j), t(ua), t(ca), t(ug), t(cg)
            s_ref = kf.kfac_precondition(ctx, J, Ua, Ca, Ug, Cg, lam, prec)
            s_new = torch.full_like(J, float("nan"))
            kf.kfac_precondition_noalloc(J, Ua, Ca, Ug, Cg, lam, prec, out=s_new, stream=ctx.stream)
            ctx.stream.synchronize()
            a, b = s_new.double().cpu().numpy(), s_ref.double().cpu().numpy()
            assert np.isfinite(a).all()
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert rel <= {"fp32": 1e-5, "tf32": 5e-3, "bf16": 2e-2}[prec], rel
