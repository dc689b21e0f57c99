"""Parity at the full one-wide-FC-layer size (A 4097 x 4097 with the bias row,
G 4096 x 4096, n = 256, s_i = i^-1.5, rho = 0.95, r = 220, p = 10, q = 1,
lambda = 0.1), the size the benchmark times, through the C-ABI with padded row
strides as the benchmark uses them.

The FP64 oracle runs the whole randomized inversion of both factors (Alg. 3
with one power iteration, Householder QR, Jacobi) on the same Omega; the
preconditioned gradient is compared on sampled columns the oracle computes one
by one (Alg. 4 restricted to those columns). Tolerances as for the FP32 path:
top-r eigenvalues to 1e-5 of lambda_1, preconditioned gradient to 1e-4
relative Frobenius (on the sampled columns).
"""
import numpy as np
import pytest

import oracle
from paper_2206_15397_gb300 import inputs
from tests import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kf():
    from paper_2206_15397_gb300 import build, kfac
    build.build()
    return kfac


@pytest.fixture(scope="module")
def ctx(kf):
    c = kf.Context(0)
    yield c
    c.close()


def padded(a: np.ndarray) -> torch.Tensor:
    """Device copy with the row stride rounded up to 4 floats (16 bytes)."""
    rows, cols = a.shape
    buf = torch.zeros((rows, (cols + 3) // 4 * 4), dtype=torch.float32, device="cuda")
    t = buf[:, :cols]
    t.copy_(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)))
    return t


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def wide_fc():
    fa, om_a = workloads.spectral(21, 4097, 230, alpha=1.5, n=256, steps=10, bias=True, use_oracle=False)
    fg, om_g = workloads.spectral(22, 4096, 230, alpha=1.5, n=256, steps=10, use_oracle=False)
    j = inputs.gradient(23, 4096, 4097, std=0.1)
    return dict(fa=fa, fg=fg, om_a=om_a, om_g=om_g, j=j, r=220, p=10, q=1, lam=0.1)


def test_wide_fc_invert_and_precondition(kf, ctx, wide_fc):
    w = wide_fc
    r, p, q, lam = w["r"], w["p"], w["q"], w["lam"]
    Ua, Da, ca = kf.kfac_rsvd_invert(ctx, padded(w["fa"]), r, p, q, lam, padded(w["om_a"]))
    Ug, Dg, cg = kf.kfac_rsvd_invert(ctx, padded(w["fg"]), r, p, q, lam, padded(w["om_g"]))
    S = kf.kfac_precondition(ctx, padded(w["j"]), Ua, ca, Ug, cg, lam)
    torch.cuda.synchronize()
    st, flags = kf.kfac_get_status(ctx)
    assert st == 0 and set(flags) <= {"CHOL_SHIFTED", "EIG_SHIFTED"}, (st, flags)

    ua, da_, ca_ = oracle.invert(w["fa"].astype(np.float64), w["om_a"].astype(np.float64), r, q, lam)
    ug, dg_, cg_ = oracle.invert(w["fg"].astype(np.float64), w["om_g"].astype(np.float64), r, q, lam)
    for D, d_o, U in ((Da, da_, Ua), (Dg, dg_, Ug)):
        err = np.abs(D.cpu().numpy().astype(np.float64) - d_o).max() / d_o[0]
        assert err <= 1e-5, err
        u = U.cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(u.T @ u, np.eye(r), atol=1e-4)

    cols = np.random.default_rng(24).choice(4097, size=24, replace=False)
    cols[0] = 4096  # the bias column
    want = oracle.precondition_cols(w["j"].astype(np.float64), ua, ca_, ug, cg_, lam, cols)
    got = S.cpu().numpy().astype(np.float64)[:, cols]
    assert rel_fro(got, want) <= 1e-4, rel_fro(got, want)
