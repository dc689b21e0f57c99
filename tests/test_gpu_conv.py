"""Conv-layer K-factors from patch statistics (kfac_ea_update_conv) against the
FP64 oracle's plain-loop patch EA update: padded and strided kernels, the bias
entry, chunked patch matrices, and the backward factor as a 1 x 1 kernel on the
output gradients; results exactly symmetric and computed on the tensor cores."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kf():
    from paper_2206_15397_gb300 import build, kfac
    build.build()
    return kfac


@pytest.mark.parametrize("shape,kernel,stride,pad,chunk", [
    ((4, 3, 16, 16), (3, 3), (1, 1), (1, 1), 0),        # first VGG16 conv: d = 28
    ((3, 8, 9, 9), (3, 2), (2, 1), (0, 1), 0),          # strided, non-square kernel
    ((5, 16, 8, 8), (3, 3), (1, 1), (1, 1), 20000),     # d = 145, one sample per chunk
])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_conv_factor_matches_oracle(kf, shape, kernel, stride, pad, chunk, prec):
    g = torch.Generator().manual_seed(sum(shape))
    x = torch.randn(*shape, generator=g)
    n, c = shape[:2]
    d = c * kernel[0] * kernel[1] + 1
    f0 = torch.randn(d, d, generator=g, dtype=torch.float64) / d
    f0 = (f0 @ f0.T).float()
    with kf.Context(0) as ctx:
        if chunk:
            kf.kfac_set_option(ctx, "conv_chunk", chunk)
        F = f0.cuda()
        n_simt = kf.kfac_simt_gemm_count()
        kf.kfac_ea_update_conv(ctx, x.cuda(), F, kernel, 0.95, stride, pad, append_one=True, prec=prec)
        assert kf.kfac_get_status(ctx)[0] == 0
        assert kf.kfac_simt_gemm_count() == n_simt
        got = F.double().cpu().numpy()
    want = oracle.ea_update_conv(f0.double().numpy(), x.double().numpy(), kernel, stride, pad, 0.95, append_one=True)
    tol = {"fp32": 2e-6, "bf16": 2e-2}[prec]
    assert np.abs(got - want).max() <= tol * np.abs(want).max()
    assert np.array_equal(got, got.T)


def test_conv_backward_factor_is_a_1x1_patch_update(kf):
    """Output gradients (n, C_out, ho, wo) with a 1 x 1 kernel and scale n: the
    per-position channel covariance of the per-sample gradients."""
    g = torch.Generator().manual_seed(7)
    go = 1e-3 * torch.randn(6, 32, 5, 5, generator=g)
    with kf.Context(0) as ctx:
        F = torch.zeros(32, 32, device="cuda")
        kf.kfac_ea_update_conv(ctx, go.cuda(), F, (1, 1), 0.9, scale=6.0)
        got = F.double().cpu().numpy()
    want = oracle.ea_update_conv(np.zeros((32, 32)), go.double().numpy(), (1, 1), rho=0.9, scale=6.0)
    assert np.abs(got - want).max() <= 2e-6 * np.abs(want).max()
