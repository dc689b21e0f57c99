"""Warm-started subspace iteration (KFAC_OPT_WARM_START, a variant beyond the
paper): after one EA step the factor moves little, so seeding the sketch with
the previous inversion's U gives the same leading eigenpairs as the oracle's
Alg. 3 on the same seed matrix [U_prev | Omega_p] (U_prev the oracle's own
previous result), and without a power iteration its rank-r approximation of
the factor carries much less error beyond the truncation error than a cold
start without one (the power iteration's products and orthonormalisation are
what the warm start saves)."""
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


@pytest.mark.parametrize("d,r,p,alpha", [(400, 40, 10, 0.8), (1025, 120, 10, 1.0)])
def test_warm_start_matches_oracle_and_saves_sweeps(kf, d, r, p, alpha):
    xs = inputs.activation_batches(91, d - 1, 96, 8, alpha=alpha, bias=True, salt=3)
    f1 = workloads.ea_factor(xs[:7]).astype(np.float32)
    f2 = workloads.ea_factor(xs).astype(np.float32)          # one more EA step
    om = inputs.omega(91, d, r + p, salt=4)
    u1_o, _ = oracle.srevd(f1.astype(np.float64), om.astype(np.float64), 1, r)
    seed = np.hstack([u1_o, om[:, :p].astype(np.float64)])
    u2_o, d2_o = oracle.srevd(f2.astype(np.float64), seed, 0, r)
    with kf.Context(0) as ctx:
        U = torch.empty(d, r, device="cuda")
        D = torch.empty(r, device="cuda")
        c = torch.empty(r, device="cuda")
        Ucold, Dcold, _ = kf.kfac_rsvd_invert(ctx, cuda(f2), r, p, 0, 0.1, cuda(om))   # cold, q = 0
        kf.kfac_rsvd_invert(ctx, cuda(f1), r, p, 1, 0.1, cuda(om), out=(U, D, c))    # previous inversion, q = 1
        kf.kfac_set_option(ctx, "warm_start", 1)
        kf.kfac_rsvd_invert(ctx, cuda(f2), r, p, 0, 0.1, cuda(om), out=(U, D, c))    # warm, q = 0
        st, flags = kf.kfac_get_status(ctx)
        assert st == 0 and set(flags) <= {"CHOL_SHIFTED", "EIG_SHIFTED"}, (st, flags)
        dd, u = D.double().cpu().numpy(), U.double().cpu().numpy()
        dcold, ucold = Dcold.double().cpu().numpy(), Ucold.double().cpu().numpy()
    assert np.abs(dd - d2_o).max() <= 1e-5 * d2_o[0]
    rec, rec_o = (u * dd) @ u.T, (u2_o * d2_o) @ u2_o.T
    assert np.linalg.norm(rec - rec_o) <= 1e-4 * np.linalg.norm(rec_o)
    f64 = f2.astype(np.float64)
    trunc = np.sqrt(np.sum(np.sort(np.linalg.eigvalsh(f64))[::-1][r:] ** 2))  # best rank-r error
    excess = lambda uu, ddv: np.linalg.norm(f64 - (uu * ddv) @ uu.T) - trunc
    assert excess(u, dd) < 0.5 * excess(ucold, dcold), (excess(u, dd), excess(ucold, dcold), trunc)
