"""RS-KFAC's inversion on the GPU (KFAC_OPT_INVERT_METHOD = 1: Alg. 2 with
power iterations, V~ and the singular values of B = Q^T F) against the FP64
oracle's Alg. 2 on the same Omega: singular values to 1e-5 of the largest,
the rank-r operator V~ diag(D) V~^T and the preconditioned gradient of
Alg. 4 to 1e-4 relative Frobenius; plus the Sec. 2.3 property that V~ sits
closer to the true leading eigenvectors than SREVD's U on the same sketch."""
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
    kf.kfac_set_option(c, "invert_method", 1)
    yield c
    c.close()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel_fro(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def check_rsvd(kf, ctx, f, om, r, p, q, lam=0.1):
    V, D, coef = kf.kfac_rsvd_invert(ctx, cuda(f), r, p, q, lam, cuda(om))
    st, flags = kf.kfac_get_status(ctx)
    assert st == 0 and set(flags) <= {"CHOL_SHIFTED", "EIG_SHIFTED"}, (st, flags)
    v_o, s_o, c_o = oracle.invert_rsvd(f.astype(np.float64), om.astype(np.float64), r, q, lam)
    v, dd = host(V), host(D)
    assert np.abs(dd - s_o).max() / s_o[0] <= 1e-5, np.abs(dd - s_o).max() / s_o[0]
    assert rel_fro((v * dd) @ v.T, (v_o * s_o) @ v_o.T) <= 1e-4
    np.testing.assert_allclose(v.T @ v, np.eye(v.shape[1]), atol=1e-4)
    # coef follows from D through Eq. (13): |dcoef| <= |dD| / lam^2
    assert np.abs(host(coef) - c_o).max() * lam * lam <= 1e-5 * s_o[0] * 10
    return V, D, coef, v_o, s_o, c_o


@pytest.mark.parametrize("d,r,p,q", [(97, 10, 6, 1), (300, 30, 10, 0), (513, 64, 10, 1), (700, 120, 20, 1)])
def test_rsvd_invert_matches_oracle(kf, ctx, d, r, p, q):
    f, om = workloads.spectral(d + 1, d, r + p, alpha=1.0 if d != 700 else 1.5, n=64, steps=6, bias=(d == 700))
    check_rsvd(kf, ctx, f, om, r, p, q)


def test_rsvd_precondition_c1(kf, ctx):
    """Config 1 end to end with RS-KFAC's V~: Alg. 4's M and S updates."""
    w = workloads.c1()
    r, p, q, lam = w["r"], w["p"], w["q"], w["lam"]
    Va, _, ca, va_o, _, ca_o = check_rsvd(kf, ctx, w["fa"], w["om_a"], r, p, q, lam)
    Vg, _, cg, vg_o, _, cg_o = check_rsvd(kf, ctx, w["fg"], w["om_g"], r, p, q, lam)
    S = kf.kfac_precondition(ctx, cuda(w["j"]), Va, ca, Vg, cg, lam)
    want = oracle.precondition(w["j"].astype(np.float64), va_o, ca_o, vg_o, cg_o, lam)
    assert rel_fro(host(S), want) <= 1e-4


def test_rsvd_v_closer_to_eigenvectors_than_srevd(kf, ctx):
    """Sec. 2.3 on the GPU: with the same Omega and no power iteration, the
    subspace of V~ is closer to the true leading r eigenvectors than SREVD's U."""
    d, r, p = 400, 20, 6
    spec = np.arange(1, d + 1, dtype=float) ** -1.0
    f64, vt, _ = inputs.low_rank_factor(61, d, spec)
    vr = vt[:, :r]
    f = cuda(f64)
    err_rsvd, err_srevd = [], []
    with kf.Context(0) as c2:
        for seed in range(6):
            om = cuda(inputs.omega(61 + seed, d, r + p))
            V, _, _ = kf.kfac_rsvd_invert(ctx, f, r, p, 0, 0.1, om)
            U, _, _ = kf.kfac_rsvd_invert(c2, f, r, p, 0, 0.1, om)
            proj = lambda m: np.linalg.norm(host(m) @ host(m).T - vr @ vr.T)
            err_rsvd.append(proj(V))
            err_srevd.append(proj(U))
    assert np.mean(err_rsvd) < 0.8 * np.mean(err_srevd), (np.mean(err_rsvd), np.mean(err_srevd))


def test_rsvd_grouped_matches_single_and_exact_path(kf, ctx):
    cases = [workloads.spectral(71, 257, 50, alpha=1.0, n=64, steps=4),
             workloads.spectral(72, 333, 50, alpha=1.5, n=64, steps=4, bias=True),
             workloads.spectral(73, 30, 50, alpha=1.0, n=16, steps=3)]   # k >= d: direct path
    items = [dict(F=cuda(f), rank=40, oversample=10, power_iters=1, lam=0.1, omega=cuda(om)) for f, om in cases]
    grouped = kf.kfac_rsvd_invert_grouped(ctx, items)
    assert kf.kfac_get_status(ctx)[0] == 0
    for it, (V, D, c) in zip(items, grouped):
        V1, D1, c1 = kf.kfac_rsvd_invert(ctx, it["F"], 40, 10, 1, 0.1, it["omega"])
        assert torch.equal(V, V1) and torch.equal(D, D1) and torch.equal(c, c1)
    f, om = cases[2]
    _, s_o, _ = oracle.invert_rsvd(f.astype(np.float64), om.astype(np.float64), 40, 1, 0.1)
    assert np.abs(host(grouped[2][1]) - s_o).max() <= 1e-5 * s_o[0]
