"""Failure detection with host-injected conditions (no GPU fault, no trap, no
hang): non-finite factors, a Jacobi sweep cap, degenerate factors (zero,
indefinite), per-item attribution in grouped calls, and the bounded waits of
the tensor-core kernels made to run out by a tiny limit. After each condition
the context stays usable and the next clean call matches the oracle."""
import numpy as np
import pytest

import oracle
from paper_2206_15397_gb300 import inputs
from tests import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KFAC_ERR_NOCONVERGE, KFAC_ERR_NONFINITE, KFAC_ERR_TIMEOUT = 5, 6, 7
BENIGN = {"CHOL_SHIFTED", "EIG_SHIFTED"}


@pytest.fixture(scope="module")
def kf():
    from paper_2206_15397_gb300 import build, kfac
    build.build()
    return kfac


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def clean_invert_matches_oracle(kf, ctx, f, om, r, p):
    U, D, c = kf.kfac_rsvd_invert(ctx, cuda(f), r, p, 1, 0.1, cuda(om))
    st, flags = kf.kfac_get_status(ctx)
    assert st == 0 and set(flags) <= BENIGN, (st, flags)
    _, d_o, _ = oracle.invert(f.astype(np.float64), om.astype(np.float64), r, 1, 0.1)
    assert np.abs(D.double().cpu().numpy() - d_o).max() <= 1e-5 * d_o[0]


def test_nonfinite_factor_is_reported_and_the_context_recovers(kf):
    f, om = workloads.spectral(51, 200, 40, alpha=1.0, n=48, steps=4)
    bad = f.copy()
    bad[3, 5] = bad[5, 3] = np.nan
    with kf.Context(0) as ctx:
        U, D, c = kf.kfac_rsvd_invert(ctx, cuda(bad), 30, 10, 1, 0.1, cuda(om))
        st, flags = kf.kfac_get_status(ctx)
        assert st == KFAC_ERR_NONFINITE and "NONFINITE" in flags, (st, flags)
        clean_invert_matches_oracle(kf, ctx, f, om, 30, 10)
        # the exact path (k >= d) checks its input too
        kf.kfac_rsvd_invert(ctx, cuda(bad[:30, :30]), 30, 10, 1, 0.1, None)
        assert kf.kfac_get_status(ctx)[0] == KFAC_ERR_NONFINITE


def test_jacobi_sweep_cap_reports_noconvergence(kf):
    f, om = workloads.spectral(52, 300, 40, alpha=1.0, n=64, steps=4)
    with kf.Context(0) as ctx:
        kf.kfac_set_option(ctx, "eig_max_sweeps", 1)
        kf.kfac_set_option(ctx, "eig_stop_tol", 0.0)   # no early stop: one sweep cannot converge
        U, D, c = kf.kfac_rsvd_invert(ctx, cuda(f), 30, 10, 1, 0.1, cuda(om))
        st, flags = kf.kfac_get_status(ctx)
        assert st == KFAC_ERR_NOCONVERGE and "EIG_NOCONV" in flags, (st, flags)
        assert all(torch.isfinite(t).all().item() for t in (U, D, c))
        kf.kfac_set_option(ctx, "eig_max_sweeps", 40)
        kf.kfac_set_option(ctx, "eig_stop_tol", 3e-3)
        clean_invert_matches_oracle(kf, ctx, f, om, 30, 10)


@pytest.mark.parametrize("d,r,p", [(200, 20, 10), (20, 16, 10)])   # sketched and exact (k >= d) paths
def test_zero_factor_gives_the_exact_damped_inverse(kf, d, r, p):
    """F = 0: every eigenvalue is 0, the coefficients vanish and the apply is
    exactly J / lambda^2 (both factors zero); the degenerate factorisations are
    flagged as shifted, not as errors."""
    lam = 0.1
    om = inputs.omega(53, d, r + p) if r + p < d else None
    with kf.Context(0) as ctx:
        F = torch.zeros(d, d, device="cuda")
        U, D, c = kf.kfac_rsvd_invert(ctx, F, r, p, 1, lam, cuda(om) if om is not None else None)
        st, flags = kf.kfac_get_status(ctx)
        assert st == 0 and set(flags) <= BENIGN, (st, flags)
        assert torch.isfinite(U).all() and D.abs().max().item() <= 1e-6 and c.abs().max().item() <= 1e-5
        j = inputs.gradient(53, d, d, std=0.1)
        S = kf.kfac_precondition(ctx, cuda(j), U, c, U, c, lam)
        assert kf.kfac_get_status(ctx)[0] == 0
        want = j.astype(np.float64) / lam ** 2
        got = S.double().cpu().numpy()
        assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)


def test_indefinite_factor_stays_finite_and_matches_the_oracle(kf):
    """A symmetric factor with negative eigenvalues (not a K-FAC factor, but a
    caller's mistake the library must survive): the eigensolver's positive
    shift grows until the factorisation succeeds, the outputs are finite and
    the Ritz values follow the oracle's."""
    d, r, p = 150, 10, 10
    spec = np.r_[np.geomspace(3.0, 1e-3, d - 3), [-0.05, -0.2, -0.4]]
    f = inputs.spectrum_factor(54, d, spec).astype(np.float32)
    om = inputs.omega(54, d, r + p)
    with kf.Context(0) as ctx:
        U, D, c = kf.kfac_rsvd_invert(ctx, cuda(f), r, p, 1, 0.1, cuda(om))
        st, flags = kf.kfac_get_status(ctx)
        assert st == 0 and set(flags) <= BENIGN, (st, flags)
        assert all(torch.isfinite(t).all().item() for t in (U, D, c))
        _, d_o, _ = oracle.invert(f.astype(np.float64), om.astype(np.float64), r, 1, 0.1)
        assert np.abs(D.double().cpu().numpy() - d_o).max() <= 1e-5 * np.abs(d_o).max()


def test_grouped_status_names_the_failing_item(kf):
    cases = [workloads.spectral(55 + i, 180, 40, alpha=1.0, n=48, steps=4) for i in range(3)]
    fs = [f.copy() for f, _ in cases]
    fs[1][7, 7] = np.inf
    items = [dict(F=cuda(f), rank=30, oversample=10, power_iters=1, lam=0.1, omega=cuda(om))
             for f, (_, om) in zip(fs, cases)]
    with kf.Context(0) as ctx:
        kf.kfac_rsvd_invert_grouped(ctx, items)
        per_item = kf.kfac_get_item_status(ctx, 3)
        assert "NONFINITE" in per_item[1], per_item
        assert set(per_item[0]) <= BENIGN and set(per_item[2]) <= BENIGN, per_item
        st, flags = kf.kfac_get_status(ctx)
        assert st == KFAC_ERR_NONFINITE and "NONFINITE" in flags
        assert kf.kfac_get_item_status(ctx, 3) == [[], [], []]   # cleared by kfac_get_status
        # the same call without the poisoned factor is clean, item by item
        items[1] = dict(items[1], F=cuda(cases[1][0]))
        kf.kfac_rsvd_invert_grouped(ctx, items)
        assert all(set(x) <= BENIGN for x in kf.kfac_get_item_status(ctx, 3))
        assert kf.kfac_get_status(ctx)[0] == 0


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
def test_tensor_core_wait_limit_runs_out_then_recovers(kf, prec):
    """With a one-cycle limit on the waits between the roles of the tensor-core
    kernels every such wait gives up: the kernel raises the timeout flag, still
    waits (with the default limit) for its own copies and tensor-core work in
    flight, and returns. The call reports KFAC_ERR_TIMEOUT; with the default
    limit restored, the same product is correct."""
    g = torch.Generator().manual_seed(56)
    A = torch.randn(256, 2048, generator=g).cuda()
    B = torch.randn(192, 2048, generator=g).cuda()
    ref = A.double() @ B.double().T
    with kf.Context(0) as ctx:
        kf.kfac_set_option(ctx, "wait_cycles", 1)
        D = torch.zeros(256, 192, device="cuda")
        kf.kfac_gemm_nt(ctx, A, B, D, prec=prec)
        st, flags = kf.kfac_get_status(ctx)
        assert st == KFAC_ERR_TIMEOUT and "TIMEOUT" in flags, (st, flags)
        assert torch.isfinite(D).all()
        kf.kfac_set_option(ctx, "wait_cycles", 4e9)
        kf.kfac_gemm_nt(ctx, A, B, D, prec=prec)
        st, flags = kf.kfac_get_status(ctx)
        assert st == 0, flags
        err = (torch.linalg.norm(D.double() - ref) / torch.linalg.norm(ref)).item()
        assert err <= {"fp32": 1e-5, "tf32": 5e-3, "bf16": 2e-2}[prec], err
