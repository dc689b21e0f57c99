"""Small single-call cases of the hot path for kernel profilers.

    python -m paper_2206_15397_gb300.profile_cases <case> [--chol-cluster]

Each case builds its inputs on the device with torch (seeded), makes a few
library calls and checks that the library reported no error, so that a
profiler can capture one kernel of a known shape with a small device
footprint (well under 1 GB):

  big_k     kfac_rsvd_invert twice on a 2048 x 2048 factor with r = 512,
            p = 10, q = 1 (k = 522: the multi-CTA Cholesky, the 17-warp
            Jacobi eigensolver, the tiled TRSM).
  k230      one inversion of a 4096 x 4096 factor with r = 220, p = 10, q = 1
            with FP32 (3xTF32) products, then the same with BF16 products.
  k230bf16  the BF16 inversion alone (BF16 copy of F read by TMA directly).
  ea_apply  the EA update of a 4096 x 4096 factor from a 4096 x 256 batch,
            then the damped Kronecker apply (Eq. 13 on both sides) of a
            4096 x 4097 gradient with r = 220 bases.

--chol-cluster factors orders above 236 on the thread-block cluster (and
solves them with the tiled kernel) instead of the blocked forms.

The factors are F = V diag(i^-2 alpha) V^T with V the Q factor of a Gaussian
matrix with min(d, m) columns (the fast-decaying spectra of Sec. 3)."""
from __future__ import annotations

import sys

import torch

from . import build, kfac


def _spectral(g, dev, d, alpha, m=640):
    v, _ = torch.linalg.qr(torch.randn(d, min(d, m), generator=g, device=dev, dtype=torch.float64))
    lam = torch.arange(1, v.shape[1] + 1, device=dev, dtype=torch.float64) ** (-2 * alpha)
    return ((v * lam) @ v.T).float().contiguous()


def run(case: str, chol_cluster: bool = False) -> None:
    build.build()
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    ctx = kfac.Context(0)
    if chol_cluster:
        kfac.kfac_set_option(ctx, "chol_blocked", 0)
    if case == "big_k":
        F = _spectral(g, dev, 2048, 1.0)
        om = torch.randn(2048, 522, generator=g, device=dev)
        for _ in range(2):
            kfac.kfac_rsvd_invert(ctx, F, 512, 10, 1, 0.1, om)
    elif case in ("k230", "k230bf16"):
        F = _spectral(g, dev, 4096, 1.5, 4096)
        om = torch.randn(4096, 230, generator=g, device=dev)
        for prec in (("fp32", "bf16") if case == "k230" else ("bf16",)):
            kfac.kfac_rsvd_invert(ctx, F, 220, 10, 1, 0.1, om, prec)
    elif case == "ea_apply":
        F = torch.zeros(4096, 4096, device=dev)
        X = torch.randn(4096, 256, generator=g, device=dev)
        kfac.kfac_ea_update(ctx, X, F, 0.95)
        J = torch.zeros(4096, 4100, device=dev)[:, :4097].normal_(generator=g)
        Ua = torch.linalg.qr(torch.randn(4097, 220, generator=g, device=dev))[0].contiguous()
        Ug = torch.linalg.qr(torch.randn(4096, 220, generator=g, device=dev))[0].contiguous()
        ca = -torch.linspace(5, 0.1, 220, device=dev)
        S = torch.zeros(4096, 4100, device=dev)[:, :4097]
        kfac.kfac_precondition(ctx, J, Ua, ca, Ug, ca, 0.1, out=S)
    else:
        raise SystemExit(f"unknown case {case!r}: big_k, k230, k230bf16, ea_apply")
    st = kfac.kfac_get_status(ctx)
    print(case, "status", st)
    if st[0] != 0:
        raise SystemExit(1)


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    run(args[0] if args else "big_k", chol_cluster="--chol-cluster" in sys.argv[1:])
