"""Batching stress: 64 factors with d ~ U{256..8192}, spectra decaying as
i^-2alpha with alpha ~ U[0.8, 2], r in {64, 128, 256, 512} capped at d, p = 10,
q = 1, inverted by one grouped call (forked streams, per-stream workspace),
then captured in a CUDA graph and replayed.

The three smallest factors are host-generated and compared with the FP64
oracle on the same Omega; every factor is checked by properties that hold at
any size: orthonormal U, descending D, Ritz values diag(U^T F U) = D. The
replayed graph reproduces the eager results bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2206_15397_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_ORACLE = 3


@pytest.fixture(scope="module")
def kf():
    from paper_2206_15397_gb300 import build, kfac
    build.build()
    return kfac


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def device_factor(gen, d, alpha):
    """F = Q diag(i^-2alpha) Q^T with Q (d x m) orthonormal from a seeded Gaussian
    (m = min(d, 640) leading directions), built with torch on the device."""
    m = min(d, 640)
    g = torch.randn(d, m, generator=gen, device="cuda", dtype=torch.float64)
    q, _ = torch.linalg.qr(g)
    w = torch.arange(1, m + 1, device="cuda", dtype=torch.float64) ** (-2.0 * alpha)
    f = (q * w) @ q.T
    return f.float().contiguous()


@pytest.fixture(scope="module")
def c5():
    shapes = inputs.batching_stress_shapes(0, 64)
    order = np.argsort([s["d"] for s in shapes])
    small = set(int(i) for i in order[:N_ORACLE])
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1234)
    items, host = [], {}
    for i, sh in enumerate(shapes):
        d, r = sh["d"], sh["r"]
        k = r + 10
        om = inputs.omega(0, d, k, salt=600 + i)
        if i in small:
            f = inputs.spectrum_factor(0, d, inputs.power_spectrum(d, 2.0 * sh["alpha"]), salt=700 + i)
            host[i] = (f.astype(np.float32), om)
            F = cuda(f)
        else:
            F = device_factor(gen, d, sh["alpha"])
        items.append(dict(F=F, rank=r, oversample=10, power_iters=1, lam=0.1, omega=cuda(om)))
    return dict(shapes=shapes, items=items, host=host)


def test_c5_grouped_invert_and_graph_replay(kf, c5):
    ctx = kf.Context(0)
    items = c5["items"]
    outs = kf.kfac_rsvd_invert_grouped(ctx, items)
    torch.cuda.synchronize()
    st, flags = kf.kfac_get_status(ctx)
    assert st == 0 and set(flags) <= {"CHOL_SHIFTED", "EIG_SHIFTED"}, (st, flags)
    # oracle on the host-generated sample
    for i, (f, om) in c5["host"].items():
        r = c5["shapes"][i]["r"]
        u_o, d_o, c_o = oracle.invert(f.astype(np.float64), om.astype(np.float64), r, 1, 0.1)
        err = np.abs(outs[i][1].cpu().numpy().astype(np.float64) - d_o).max() / d_o[0]
        assert err <= 1e-5, (i, err)
    # properties of every factor
    for i, (U, D, _) in enumerate(outs):
        u = U.double()
        r = u.shape[1]
        assert (u.T @ u - torch.eye(r, device="cuda", dtype=torch.float64)).abs().max().item() <= 1e-4, i
        dd = D.double()
        assert torch.all(dd[:-1] >= dd[1:]).item(), i
        ritz = torch.diagonal(u.T @ items[i]["F"].double() @ u)
        assert ((ritz - dd).abs().max() / dd[0]).item() <= 1e-5, i
    # graph capture of the same grouped call, writing into the eager outputs' buffers copies
    ref = [tuple(t.clone() for t in o) for o in outs]
    gitems = [dict(it, out=o) for it, o in zip(items, outs)]
    for o in outs:
        for t in o:
            t.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        ctx.set_stream(torch.cuda.current_stream())
        kf.kfac_rsvd_invert_grouped(ctx, gitems)
    ctx.set_stream(torch.cuda.current_stream())
    graph.replay()
    torch.cuda.synchronize()
    assert kf.kfac_get_status(ctx)[0] == 0
    for a, b in zip(ref, outs):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    ctx.close()
