"""The seed path of the inversion: the library draws the Gaussian test matrix on
the device (Philox4x32-10 + Box-Muller in FP32) when omega is NULL. The draw is
checked against the host generator's FP64 evaluation of the same formula, the
seeded inversion against the oracle fed with that host matrix, and against the
same call with the drawn matrix passed explicitly (bitwise)."""
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


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("d,k,seed", [(1, 1, 0), (7, 3, 5), (257, 74, 2024), (1000, 230, (7 << 32) + 3),
                                      (4097, 522, 99)])
def test_draw_matches_host_definition(kf, ctx, d, k, seed):
    got = host(kf.kfac_draw_omega(ctx, d, k, seed))
    want = inputs.seeded_omega(seed, d, k).astype(np.float64)
    err = np.abs(got - want) / (1.0 + np.abs(want))
    assert err.max() <= 1e-6, err.max()
    st, flags = kf.kfac_get_status(ctx)
    assert st == 0 and not flags


def test_draw_into_strided_buffer(kf, ctx):
    base = torch.full((300, 80), 7.0, device="cuda")
    kf.kfac_draw_omega(ctx, 300, 74, 3, out=base[:, :74])
    np.testing.assert_array_equal(host(base[:, 74:]), 7.0)   # the pad columns untouched
    np.testing.assert_array_equal(host(base[:, :74]), host(kf.kfac_draw_omega(ctx, 300, 74, 3)))


@pytest.mark.parametrize("d,r,p,q,seed", [(97, 10, 6, 1, 1), (513, 64, 10, 1, 77), (700, 120, 10, 2, 12345)])
def test_seeded_invert_matches_explicit_and_oracle(kf, ctx, d, r, p, q, seed):
    f, _ = workloads.spectral(d, d, r + p, alpha=1.0, n=48, steps=6)
    k = r + p
    F = cuda(f)
    U, D, c = kf.kfac_rsvd_invert(ctx, F, r, p, q, 0.1, None, seed=seed)
    om = kf.kfac_draw_omega(ctx, d, k, seed)
    U2, D2, c2 = kf.kfac_rsvd_invert(ctx, F, r, p, q, 0.1, om)
    assert torch.equal(U, U2) and torch.equal(D, D2) and torch.equal(c, c2)
    st, flags = kf.kfac_get_status(ctx)
    assert st == 0 and set(flags) <= {"CHOL_SHIFTED", "EIG_SHIFTED"}, (st, flags)
    u_o, d_o, _ = oracle.invert(f.astype(np.float64), inputs.seeded_omega(seed, d, k).astype(np.float64), r, q, 0.1)
    dd, u = host(D), host(U)
    assert np.abs(dd - d_o).max() / d_o[0] <= 1e-5
    rec, rec_o = (u * dd) @ u.T, (u_o * d_o) @ u_o.T
    assert np.linalg.norm(rec - rec_o) / np.linalg.norm(rec_o) <= 1e-4
    # another seed gives another sketch (different rounding, same spectrum)
    U3, D3, _ = kf.kfac_rsvd_invert(ctx, F, r, p, q, 0.1, None, seed=seed + 1)
    assert not torch.equal(U3, U)


def test_seeded_grouped_and_warm_start(kf, ctx):
    shapes = [(300, 40, 10), (130, 20, 6), (513, 64, 10)]
    fs = [workloads.spectral(i + 3, d, r + p, alpha=1.2, n=32, steps=4)[0] for i, (d, r, p) in enumerate(shapes)]
    items = [dict(F=cuda(f), rank=r, oversample=p, power_iters=1, lam=0.1, omega=None, seed=10 + i)
             for i, (f, (d, r, p)) in enumerate(zip(fs, shapes))]
    outs = kf.kfac_rsvd_invert_grouped(ctx, items)
    for it, (U, D, c) in zip(items, outs):
        U1, D1, c1 = kf.kfac_rsvd_invert(ctx, it["F"], it["rank"], it["oversample"], 1, 0.1, None, seed=it["seed"])
        assert torch.equal(U, U1) and torch.equal(D, D1) and torch.equal(c, c1)
    # warm start: [U_prev | first k - r columns of the seeded matrix]
    kf.kfac_set_option(ctx, "warm_start", 1)
    try:
        d, r, p = shapes[2]
        F = items[2]["F"]
        prev = outs[2][0].clone()
        Ua, Da, _ = kf.kfac_rsvd_invert(ctx, F, r, p, 1, 0.1, None, out=(prev.clone(), torch.empty(r, device="cuda"),
                                                                        torch.empty(r, device="cuda")), seed=5)
        Ub, Db, _ = kf.kfac_rsvd_invert(ctx, F, r, p, 1, 0.1, kf.kfac_draw_omega(ctx, d, r + p, 5),
                                        out=(prev.clone(), torch.empty(r, device="cuda"), torch.empty(r, device="cuda")))
        assert torch.equal(Ua, Ub) and torch.equal(Da, Db)
    finally:
        kf.kfac_set_option(ctx, "warm_start", 0)
    st, flags = kf.kfac_get_status(ctx)
    assert st == 0 and set(flags) <= {"CHOL_SHIFTED", "EIG_SHIFTED"}, (st, flags)
