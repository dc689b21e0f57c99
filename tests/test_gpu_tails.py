"""Precomputed 3xTF32 tails (KFAC_OPT_TAIL_PLANES = 1, the default) against
tails formed per tile in shared memory (= 0): the tails are the same function
of the same values either way, so every FP32 result must be bitwise equal -
inversion (SREVD and RSVD, single and grouped), EA updates (column batches,
row batches, conv patches) and the preconditioner apply, on ragged shapes."""
import numpy as np
import pytest

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


def both(kf, fn, **opts):
    """fn(ctx) with tail planes on, then off; returns the two results."""
    out = []
    for tails in (1, 0):
        with kf.Context(0) as ctx:
            kf.kfac_set_option(ctx, "tail_planes", tails)
            for k, v in opts.items():
                kf.kfac_set_option(ctx, k, v)
            res = fn(ctx)
            st, flags = kf.kfac_get_status(ctx)
            assert st == 0 and set(flags) <= {"CHOL_SHIFTED", "EIG_SHIFTED"}, (st, flags)
            out.append([t.clone() for t in res])
    return out


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("d,r,p", [(700, 120, 10), (1031, 250, 10)])
def test_inversion_bitwise(kf, method, d, r, p):
    f, om = workloads.spectral(90 + d, d, r + p, alpha=1.2, n=64, steps=4, bias=(d == 1031))
    F, Om = cuda(f), cuda(om)
    on, off = both(kf, lambda ctx: kf.kfac_rsvd_invert(ctx, F, r, p, 1, 0.1, Om), invert_method=method)
    for a, b in zip(on, off):
        assert torch.equal(a, b)


def test_grouped_inversion_bitwise(kf):
    cases = [workloads.spectral(95 + i, d, 60, alpha=1.0, n=64, steps=3) for i, d in enumerate((257, 402, 333))]
    items = [dict(F=cuda(f), rank=50, oversample=10, power_iters=1, lam=0.1, omega=cuda(om)) for f, om in cases]
    on, off = both(kf, lambda ctx: [t for it in kf.kfac_rsvd_invert_grouped(ctx, items) for t in it])
    for a, b in zip(on, off):
        assert torch.equal(a, b)


def test_ea_updates_bitwise(kf):
    d, n = 517, 203
    x = cuda(inputs.gaussian(97, (d, n)))
    f0 = cuda(inputs.spectrum_factor(97, d, inputs.power_spectrum(d, 1.0)))
    rows = cuda(inputs.gaussian(98, (n, d - 1)))
    img = cuda(inputs.gaussian(99, (3, 7, 12, 11)))

    def run(ctx):
        F1 = f0.clone()
        kf.kfac_ea_update(ctx, x, F1, 0.9)
        F2 = f0.clone()
        kf.kfac_ea_update_rows(ctx, rows, F2, 0.9, append_one=True, scale=2.0)
        F3 = torch.zeros(7 * 9 + 1, 7 * 9 + 1, device="cuda")
        kf.kfac_ea_update_conv(ctx, img, F3, (3, 3), 0.0, stride=(1, 1), padding=(1, 1), append_one=True)
        return F1, F2, F3

    on, off = both(kf, run)
    for a, b in zip(on, off):
        assert torch.equal(a, b)


def test_apply_bitwise(kf):
    dg, da, ra, rg = 301, 517, 90, 70
    j = cuda(inputs.gradient(100, dg, da, std=0.1))
    Ua = torch.linalg.qr(cuda(inputs.gaussian(101, (da, ra))))[0].contiguous()
    Ug = torch.linalg.qr(cuda(inputs.gaussian(102, (dg, rg))))[0].contiguous()
    ca = -torch.linspace(5, 0.1, ra, device="cuda")
    cg = -torch.linspace(3, 0.2, rg, device="cuda")
    on, off = both(kf, lambda ctx: [kf.kfac_precondition(ctx, j, Ua, ca, Ug, cg, 0.1)])
    assert torch.equal(on[0], off[0])


def test_gemm_nt_bitwise(kf):
    A = cuda(inputs.gaussian(103, (333, 1029)))
    B = cuda(inputs.gaussian(104, (522, 1029)))
    on, off = both(kf, lambda ctx: [kf.kfac_gemm_nt(ctx, A, B, torch.zeros(333, 522, device="cuda"))])
    assert torch.equal(on[0], off[0])
