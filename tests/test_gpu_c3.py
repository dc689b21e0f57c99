"""The VGG16_bn factor set (13 conv layers and the FC layer: A factors
C_in*9+1 = 28 ... 4609 and 513, G factors 64 ... 512 and 10; n = 128, 10 EA
steps, r = min(d, 220), p = 10, q = 1, lambda = 0.1), all 28 factors inverted
by one grouped call and all 14 layers preconditioned by another.

FP32 path: the FP64 oracle inverts a fixed sample of factors on the same Omega
(the exact path d <= k included) and the preconditioned gradient is compared
on sampled columns of the layers whose two factors are both in the sample;
the 4609-wide factors are checked by properties that hold at any size
(orthonormal U, descending D, Ritz values diag(U^T F U) = D).
Precision form (TF32 / BF16 operands, FP32 accumulation, FP64 Cholesky and
eigensolve): the same comparisons at the reduced-precision tolerance 2e-2,
with the per-factor errors printed.
"""
import numpy as np
import pytest

import oracle
from tests import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SAMPLE_LAYERS = (0, 2, 4, 7, 13)  # A 28 (exact) / G 64 (exact), 577 / 128, 1153 / 256, 2305 / 512, 513 / 10
TOL = {"fp32": (1e-5, 1e-4), "tf32": (2e-2, 2e-2), "bf16": (2e-2, 2e-2)}


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


@pytest.fixture(scope="module")
def c3():
    w = workloads.c3()
    lam, q = w["lam"], w["q"]
    ref = {}
    for li in SAMPLE_LAYERS:
        L = w["layers"][li]
        for side in ("a", "g"):
            f = L["f" + side].astype(np.float64)
            r = L["r_" + side]
            ref[(li, side)] = oracle.invert(f, L["om_" + side].astype(np.float64), r, q, lam)
    w["ref"] = ref
    return w


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def run_c3(kf, ctx, w, prec):
    p, q, lam = w["p"], w["q"], w["lam"]
    items = []
    for L in w["layers"]:
        for side in ("a", "g"):
            items.append(dict(F=cuda(L["f" + side]), rank=L["r_" + side], oversample=p, power_iters=q, lam=lam,
                              omega=cuda(L["om_" + side]), prec=prec))
    n_simt = kf.kfac_simt_gemm_count()
    outs = kf.kfac_rsvd_invert_grouped(ctx, items)
    pitems = []
    for li, L in enumerate(w["layers"]):
        (Ua, _, ca), (Ug, _, cg) = outs[2 * li], outs[2 * li + 1]
        pitems.append(dict(J=cuda(L["j"]), U_a=Ua, coef_a=ca, U_g=Ug, coef_g=cg, lam=lam, prec=prec))
    S = kf.kfac_precondition_grouped(ctx, pitems)
    torch.cuda.synchronize()
    st, flags = kf.kfac_get_status(ctx)
    assert st == 0 and set(flags) <= {"CHOL_SHIFTED", "EIG_SHIFTED"}, (st, flags)
    # unpadded tensors (A factors 28 ... 4609 wide): every product on the tensor cores
    assert kf.kfac_simt_gemm_count() == n_simt
    return items, outs, S


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
def test_c3_grouped_invert_and_precondition(kf, ctx, c3, prec):
    eig_tol, s_tol = TOL[prec]
    items, outs, S = run_c3(kf, ctx, c3, prec)
    lam = c3["lam"]
    report = []
    for li in SAMPLE_LAYERS:
        L = c3["layers"][li]
        for side, idx in (("a", 2 * li), ("g", 2 * li + 1)):
            u_o, d_o, c_o = c3["ref"][(li, side)]
            U, D, coef = outs[idx]
            err = np.abs(D.cpu().numpy().astype(np.float64) - d_o).max() / d_o[0]
            report.append((li, side, L["f" + side].shape[0], err))
            assert err <= eig_tol, (li, side, err)
        (ua, _, ca), (ug, _, cg) = c3["ref"][(li, "a")], c3["ref"][(li, "g")]
        da = L["fa"].shape[0]
        cols = np.unique(np.r_[np.random.default_rng(li).choice(da, size=min(da, 12), replace=False), da - 1])
        want = oracle.precondition_cols(L["j"].astype(np.float64), ua, ca, ug, cg, lam, cols)
        got = S[li].cpu().numpy().astype(np.float64)[:, cols]
        rel = np.linalg.norm(got - want) / np.linalg.norm(want)
        report.append((li, "S", da, rel))
        assert rel <= s_tol, (li, rel)
    print(f"\n[{prec}] per-factor |dD|/D1 and sampled-S relative errors vs the FP64 oracle:")
    for li, side, d, e in report:
        print(f"  layer {li:2d} {side} d={d:5d}: {e:.2e}")
    # the wide factors: properties at any size
    for li in range(len(c3["layers"])):
        if li in SAMPLE_LAYERS:
            continue
        for side, idx in (("a", 2 * li), ("g", 2 * li + 1)):
            U, D, _ = outs[idx]
            F = items[idx]["F"].double()
            u = U.double()
            r = u.shape[1]
            orth = (u.T @ u - torch.eye(r, device=u.device, dtype=torch.float64)).abs().max().item()
            assert orth <= (1e-4 if prec == "fp32" else 2e-2), (li, side, orth)
            dd = D.double()
            assert torch.all(dd[:-1] >= dd[1:]).item()
            ritz = torch.diagonal(u.T @ F @ u)
            assert ((ritz - dd).abs().max() / dd[0]).item() <= eig_tol * 10, (li, side)


def test_grouped_ea_matches_single_calls(kf, ctx):
    from paper_2206_15397_gb300 import inputs
    rng_dims = [(37, 16), (300, 64), (129, 33)]
    xs = [cuda(inputs.gradient(7, d, n, std=1.0, salt=i)) for i, (d, n) in enumerate(rng_dims)]
    f0 = [cuda(np.eye(d) * 0.5) for d, _ in rng_dims]
    single = [f.clone() for f in f0]
    for x, f in zip(xs, single):
        kf.kfac_ea_update(ctx, x, f, 0.9)
    grouped = [f.clone() for f in f0]
    kf.kfac_ea_update_grouped(ctx, [dict(X=x, F=f, rho=0.9) for x, f in zip(xs, grouped)])
    torch.cuda.synchronize()
    for a, b in zip(single, grouped):
        assert torch.equal(a, b)


def test_grouped_precondition_matches_single_calls(kf, ctx):
    from paper_2206_15397_gb300 import inputs
    shapes = [(64, 577, 40, 30), (10, 513, 10, 8), (256, 1153, 200, 100)]
    items, single = [], []
    for i, (dg, da, ra, rg) in enumerate(shapes):
        J = cuda(inputs.gradient(8, dg, da, std=0.1, salt=i))
        Ua, _ = torch.linalg.qr(cuda(inputs.gradient(8, da, ra, std=1.0, salt=10 + i)))
        Ug, _ = torch.linalg.qr(cuda(inputs.gradient(8, dg, rg, std=1.0, salt=20 + i)))
        ca = -torch.linspace(5.0, 0.1, ra, device="cuda")
        cg = -torch.linspace(3.0, 0.2, rg, device="cuda")
        Ua, Ug = Ua.contiguous(), Ug.contiguous()
        single.append(kf.kfac_precondition(ctx, J, Ua, ca, Ug, cg, 0.1))
        items.append(dict(J=J, U_a=Ua, coef_a=ca, U_g=Ug, coef_g=cg, lam=0.1))
    grouped = kf.kfac_precondition_grouped(ctx, items)
    torch.cuda.synchronize()
    for a, b in zip(single, grouped):
        assert torch.equal(a, b)
