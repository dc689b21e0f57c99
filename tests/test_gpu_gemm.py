"""The GEMM engine under the entry points (the tcgen05 tensor-core kernels;
operands whose rows TMA cannot address are first copied with a padded stride),
through the kfac_gemm_nt utility of the C ABI, against FP64 products.
Tolerances: FP32-accurate 3xTF32 1e-5, TF32 5e-3 and BF16 2e-2 relative
Frobenius."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "tf32": 5e-3, "bf16": 2e-2}


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


def padded(rows, cols, pad, seed):
    """(rows, cols) view of a (rows, cols + pad) CUDA tensor: row stride cols + pad."""
    g = torch.Generator().manual_seed(seed)
    base = torch.randn(rows, cols + pad, generator=g, dtype=torch.float32)
    return base.cuda()[:, :cols]


@pytest.mark.parametrize("M,N,K,pad", [
    (128, 128, 32, 0),       # one tile, one K block
    (256, 256, 256, 0),
    (130, 230, 97, 3),       # ragged M, N, K; row strides 100 / 100 floats
    (1000, 230, 4097, 3),    # few tiles, long K: split-K with the reducing epilogue
    (300, 64, 1024, 0),
    (77, 5, 9, 0),           # K not a multiple of 4: operands copied to a padded stride
    (65, 33, 577, 0),        # row stride 577 floats (a VGG16 conv factor's width)
])
@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
def test_gemm_nt(kf, ctx, M, N, K, pad, prec):
    A = padded(M, K, pad, 1)
    B = padded(N, K, pad, 2)
    D0 = torch.randn(M, N, device="cuda")
    D = D0.clone()
    n_simt = kf.kfac_simt_gemm_count()
    kf.kfac_gemm_nt(ctx, A, B, D, alpha=0.7, beta=0.3, prec=prec)
    assert kf.kfac_simt_gemm_count() == n_simt   # every stride runs on the tensor cores
    ref = 0.7 * (A.double() @ B.double().T) + 0.3 * D0.double()
    st, flags = kf.kfac_get_status(ctx)
    assert st == 0, flags
    err = (torch.linalg.norm(D.double() - ref) / torch.linalg.norm(ref)).item()
    assert err <= TOL[prec], err


def test_gemm_nt_zero_k(kf, ctx):
    A = torch.zeros(8, 0, device="cuda")
    D = torch.ones(8, 8, device="cuda")
    kf.kfac_gemm_nt(ctx, A, torch.zeros(8, 0, device="cuda"), D, alpha=1.0, beta=2.0)
    assert torch.equal(D, torch.full_like(D, 2.0))


@pytest.mark.parametrize("M,N,K,pad", [
    (128, 128, 64, 0),       # one tile, one BF16 K-step
    (130, 230, 97, 3),       # ragged M, N, K (K-step 64 with a zero-filled tail)
    (1000, 230, 4097, 3),    # split-K into 64-aligned chunks
    (256, 384, 1000, 0),
])
def test_gemm_nt_bf16_exact_operands(kf, ctx, M, N, K, pad):
    """BF16 operand path: each operand is rounded to nearest BF16 and the
    products are summed in FP32, so against the FP64 product of the rounded
    operands only FP32 accumulation error remains (a wrong rounding mode, a
    mis-swizzled K-chunk or a dropped K-step shows up far above 2e-5)."""
    A = padded(M, K, pad, 11)
    B = padded(N, K, pad, 12)
    D = torch.zeros(M, N, device="cuda")
    kf.kfac_gemm_nt(ctx, A, B, D, alpha=1.0, beta=0.0, prec="bf16")
    st, flags = kf.kfac_get_status(ctx)
    assert st == 0, flags
    ref = A.bfloat16().double() @ B.bfloat16().double().T
    err = (torch.linalg.norm(D.double() - ref) / torch.linalg.norm(ref)).item()
    assert err <= 2e-5, err
