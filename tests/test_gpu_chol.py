"""Large-order Cholesky factorisations (sketch widths k above the one-CTA
kernel's 236) and the CholeskyQR solves: the blocked factorisation
(KFAC_OPT_CHOL_BLOCKED = 1, the default) or the cluster kernel (= 0), with the
solves through the explicit inverse (KFAC_OPT_TRSM_INVERSE = 1, the default)
or by substitution (= 0), each give inversions that match the FP64 oracle
(Alg. 3: eigenvalues to 1e-5 of the largest, orthonormal U, Alg. 4's
preconditioned gradient), for the CholeskyQR Grams and the eigensolver's
factor alike; degenerate inputs (zero, non-finite) take the failure paths."""
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


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("blocked,inverse", [(1, 1), (1, 0), (0, 0)])
@pytest.mark.parametrize("d,r,alpha", [(700, 256, 1.0), (1100, 512, 1.5), (560, 560, 1.0)])
def test_large_k_inversion_matches_oracle(kf, blocked, inverse, d, r, alpha):
    """k = 266, 522 (sketched) and d = 560 <= k (exact path: the eigensolver
    factors the whole factor)."""
    p, lam = 10, 0.1
    f, om = workloads.spectral(110 + d, d, min(r + p, d), alpha=alpha, n=96, steps=6, bias=(d == 1100))
    om_t = cuda(om) if r + p < d else None
    if r + p >= d:
        om = None
    with kf.Context(0) as ctx:
        kf.kfac_set_option(ctx, "chol_blocked", blocked)
        kf.kfac_set_option(ctx, "trsm_inverse", inverse)
        U, D, c = kf.kfac_rsvd_invert(ctx, cuda(f), r, p, 1, lam, om_t)
        st, flags = kf.kfac_get_status(ctx)
        assert st == 0 and set(flags) <= {"CHOL_SHIFTED", "EIG_SHIFTED"}, (st, flags)
        om_o = om.astype(np.float64) if r + p < d else np.zeros((d, r + p))
        u_o, d_o, c_o = oracle.invert(f.astype(np.float64), om_o, r, 1, lam)
        dd = host(D)
        assert np.abs(dd - d_o).max() <= 1e-5 * d_o[0], np.abs(dd - d_o).max() / d_o[0]
        u = host(U)
        np.testing.assert_allclose(u.T @ u, np.eye(u.shape[1]), atol=2e-5)
        # Alg. 4 with this factor on the A side and a fixed small G side
        j = inputs.gradient(111, 64, d, std=0.1)
        ug = np.linalg.qr(inputs.gaussian(114, (64, 8)))[0]
        cg = -np.linspace(3.0, 0.5, 8)
        S = kf.kfac_precondition(ctx, cuda(j), U, c, cuda(ug), cuda(cg), lam)
        assert kf.kfac_get_status(ctx)[0] == 0
        want = oracle.precondition(j.astype(np.float64), u_o, c_o, ug.astype(np.float32).astype(np.float64),
                                   cg.astype(np.float32).astype(np.float64), lam)
        assert np.linalg.norm(host(S) - want) <= 1e-4 * np.linalg.norm(want)


@pytest.mark.parametrize("blocked,inverse", [(1, 1), (0, 0)])
def test_large_k_zero_and_nonfinite_factors(kf, blocked, inverse):
    d, r, p = 600, 300, 10
    om = cuda(inputs.omega(112, d, r + p))
    with kf.Context(0) as ctx:
        kf.kfac_set_option(ctx, "chol_blocked", blocked)
        kf.kfac_set_option(ctx, "trsm_inverse", inverse)
        U, D, c = kf.kfac_rsvd_invert(ctx, torch.zeros(d, d, device="cuda"), r, p, 1, 0.1, om)
        st, flags = kf.kfac_get_status(ctx)
        assert st == 0 and set(flags) <= {"CHOL_SHIFTED", "EIG_SHIFTED"}, (st, flags)
        assert torch.isfinite(U).all() and D.abs().max().item() <= 1e-6 and c.abs().max().item() <= 1e-5
        f, _ = workloads.spectral(113, d, r + p, alpha=1.0, n=64, steps=4)
        f[10, 20] = f[20, 10] = np.nan
        kf.kfac_rsvd_invert(ctx, cuda(f), r, p, 1, 0.1, om)
        st, flags = kf.kfac_get_status(ctx)
        assert st != 0 and "NONFINITE" in flags, (st, flags)


@pytest.mark.parametrize("inverse", [1, 0])
def test_steep_spectrum_blocked_factorisations_do_not_break_down(kf, inverse):
    """A k = 522 sketch of a factor whose eigenvalues fall as i^-3.6 over 640
    directions (the steepest of the batching-stress set): the sketch is
    numerically rank-deficient from about the 80th column, and the blocked
    Cholesky of the CholeskyQR Grams once overflowed in a diagonal block on some
    test matrices. Over many seeded draws every inversion must succeed (a block
    that overflows is retried with a shift of its own), with orthonormal U and
    the leading eigenvalues of the factor."""
    d, m, r, p, lam = 3238, 640, 512, 10, 0.1
    gen = torch.Generator(device="cuda")
    gen.manual_seed(19)
    v, _ = torch.linalg.qr(torch.randn(d, m, generator=gen, device="cuda", dtype=torch.float64))
    s2 = torch.arange(1, m + 1, device="cuda", dtype=torch.float64) ** (-3.63)
    F = ((v * s2) @ v.T).float()
    lam_ref = s2[:r].cpu().numpy()
    with kf.Context(0) as ctx:
        kf.kfac_set_option(ctx, "trsm_inverse", inverse)
        for seed in range(12):
            U, D, _ = kf.kfac_rsvd_invert(ctx, F, r, p, 1, lam, None, seed=1000 + seed)
            st, flags = kf.kfac_get_status(ctx)
            assert st == 0 and set(flags) <= {"CHOL_SHIFTED", "EIG_SHIFTED"}, (seed, st, flags)
            u = U.double()
            assert (u.T @ u - torch.eye(r, device="cuda", dtype=torch.float64)).abs().max().item() <= 1e-4, seed
            assert np.abs(host(D) - lam_ref).max() <= 1e-5 * lam_ref[0], seed
