"""CUDA-graph capture of a whole K-factor step (grouped EA update, grouped
randomized inversion on forked streams, grouped preconditioner apply): once an
eager call has sized the workspace and created the side streams, the same calls
record into a graph without allocating, and replays reproduce the eager
results bit for bit (also after the inputs change in place)."""
import numpy as np
import pytest

from paper_2206_15397_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kf():
    from paper_2206_15397_gb300 import build, kfac
    build.build()
    return kfac


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def make_step(kf, ctx, bufs):
    """One step: EA of both factors, grouped inversion, precondition; every
    output goes to a preallocated buffer."""
    kf.kfac_ea_update_grouped(ctx, [dict(X=bufs["xa"], F=bufs["fa"], rho=0.95),
                                    dict(X=bufs["xg"], F=bufs["fg"], rho=0.95)])
    kf.kfac_rsvd_invert_grouped(ctx, [
        dict(F=bufs["fa"], rank=40, oversample=10, power_iters=1, lam=0.1, omega=bufs["oa"], out=bufs["inv_a"]),
        dict(F=bufs["fg"], rank=30, oversample=10, power_iters=1, lam=0.1, omega=bufs["og"], out=bufs["inv_g"])])
    (Ua, _, ca), (Ug, _, cg) = bufs["inv_a"], bufs["inv_g"]
    kf.kfac_precondition_grouped(ctx, [dict(J=bufs["j"], U_a=Ua, coef_a=ca, U_g=Ug, coef_g=cg, lam=0.1,
                                            out=bufs["s"])])


def test_step_captures_and_replays_bitwise(kf):
    da, dg, n = 513, 300, 64
    xa = inputs.activation_batches(5, da - 1, n, 2, alpha=1.0, bias=True, salt=1)
    xg = inputs.activation_batches(5, dg, n, 2, alpha=1.0, salt=2)
    bufs = dict(xa=cuda(xa[0]), xg=cuda(xg[0]), fa=torch.zeros(da, da, device="cuda"),
                fg=torch.zeros(dg, dg, device="cuda"), oa=cuda(inputs.omega(5, da, 50, salt=3)),
                og=cuda(inputs.omega(5, dg, 40, salt=4)), j=cuda(inputs.gradient(5, dg, da, std=0.1)),
                s=torch.empty(dg, da, device="cuda"))
    bufs["inv_a"] = (torch.empty(da, 40, device="cuda"), torch.empty(40, device="cuda"), torch.empty(40, device="cuda"))
    bufs["inv_g"] = (torch.empty(dg, 30, device="cuda"), torch.empty(30, device="cuda"), torch.empty(30, device="cuda"))
    ctx = kf.Context(0)
    # eager: two steps (the second sees a non-zero factor) -> reference results
    fa0, fg0 = bufs["fa"].clone(), bufs["fg"].clone()
    make_step(kf, ctx, bufs)
    bufs["xa"].copy_(cuda(xa[1])); bufs["xg"].copy_(cuda(xg[1]))
    make_step(kf, ctx, bufs)
    torch.cuda.synchronize()
    assert kf.kfac_get_status(ctx)[0] == 0
    ref = [t.clone() for t in (bufs["fa"], bufs["fg"], bufs["s"], *bufs["inv_a"], *bufs["inv_g"])]
    # capture one step, replay twice from the same starting state
    bufs["fa"].copy_(fa0); bufs["fg"].copy_(fg0); bufs["xa"].copy_(cuda(xa[0])); bufs["xg"].copy_(cuda(xg[0]))
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        ctx.set_stream(torch.cuda.current_stream())
        make_step(kf, ctx, bufs)
    ctx.set_stream(torch.cuda.current_stream())
    graph.replay()
    bufs["xa"].copy_(cuda(xa[1])); bufs["xg"].copy_(cuda(xg[1]))
    graph.replay()
    torch.cuda.synchronize()
    assert kf.kfac_get_status(ctx)[0] == 0
    got = [bufs["fa"], bufs["fg"], bufs["s"], *bufs["inv_a"], *bufs["inv_g"]]
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    ctx.close()


def test_stage_profile_and_timeline(kf):
    """The stage profiler: per-stage totals equal the sum of the timeline's
    intervals, grouped items are tagged with their index, and every interval
    lies inside the host-measured span of the call."""
    cases = [(257, 30), (300, 20), (140, 40)]
    items = []
    for i, (d, r) in enumerate(cases):
        f = inputs.spectrum_factor(80 + i, d, inputs.power_spectrum(d, 1.0) ** 2).astype(np.float32)
        items.append(dict(F=cuda(f), rank=r, oversample=10, power_iters=1, lam=0.1,
                          omega=cuda(inputs.omega(80 + i, d, r + 10))))
    with kf.Context(0) as ctx:
        kf.kfac_rsvd_invert_grouped(ctx, items)    # sizes the workspace, creates the side streams
        torch.cuda.synchronize()
        kf.kfac_profile_enable(ctx, True)
        kf.kfac_rsvd_invert_grouped(ctx, items)
        tl = kf.kfac_profile_timeline(ctx)
        tot = kf.kfac_profile_read(ctx)
        kf.kfac_profile_enable(ctx, False)
        assert kf.kfac_get_status(ctx)[0] == 0
    assert tl and {it for _, it, _, _ in tl} == {0, 1, 2}
    assert all(0.0 <= a <= b for _, _, a, b in tl)
    assert [a for _, _, a, _ in tl] == sorted(a for _, _, a, _ in tl)
    for name, (ms, n) in tot.items():
        iv = [(a, b) for s, _, a, b in tl if s == name]
        assert len(iv) == n
        assert abs(sum(b - a for a, b in iv) - ms) <= 1e-3 * max(ms, 1.0)
    for stage in ("sketch_gemm", "cholqr_chol", "eig_jacobi", "lift_gemm"):
        assert {it for s, it, _, _ in tl if s == stage} == {0, 1, 2}, stage


def test_fused_step_matches_the_three_grouped_calls(kf):
    """kfac_step_grouped (per-item dependencies, applies overlapping the
    inversions) gives bitwise the results of the grouped EA, inversion and
    apply calls in turn, eagerly and replayed from a CUDA graph."""
    dims = [(513, 40), (300, 30), (257, 50), (120, 20), (700, 60), (64, 70)]   # (d, r); the last is exact
    layers = [(0, 1), (2, 3), (4, 5)]
    n = 48

    def state():
        st = dict(F=[], X=[], O=[], out=[], J=[], S=[])
        for i, (d, r) in enumerate(dims):
            st["F"].append(cuda(inputs.spectrum_factor(90 + i, d, inputs.power_spectrum(d, 1.0) ** 2)))
            st["X"].append(cuda(inputs.gaussian(120 + i, (d, n))))
            k = r + 10
            st["O"].append(cuda(inputs.omega(90 + i, d, k)) if k < d else None)
            st["out"].append((torch.empty(d, min(r, d), device="cuda"), torch.empty(min(r, d), device="cuda"),
                              torch.empty(min(r, d), device="cuda")))
        for a, g in layers:
            st["J"].append(cuda(inputs.gradient(95 + a, dims[g][0], dims[a][0], std=0.1)))
            st["S"].append(torch.empty(dims[g][0], dims[a][0], device="cuda"))
        return st

    def descs(st):
        ea = kf.ea_descs([dict(X=st["X"][i], F=st["F"][i], rho=0.9) for i in range(len(dims))])
        inv, _ = kf.invert_descs([dict(F=st["F"][i], rank=r, oversample=10, power_iters=1, lam=0.1,
                                       omega=st["O"][i], out=st["out"][i]) for i, (d, r) in enumerate(dims)])
        pre, _ = kf.precond_descs([dict(J=st["J"][li], U_a=st["out"][a][0], coef_a=st["out"][a][2],
                                        U_g=st["out"][g][0], coef_g=st["out"][g][2], lam=0.1, out=st["S"][li])
                                   for li, (a, g) in enumerate(layers)])
        return ea, inv, pre

    def outputs(st):
        return [t.clone() for t in st["F"] + [u for o in st["out"] for u in o] + st["S"]]

    ref_st = state()
    ea, inv, pre = descs(ref_st)
    with kf.Context(0) as ctx:
        kf.call_grouped(ctx, "ea", ea)
        kf.call_grouped(ctx, "invert", inv)
        kf.call_grouped(ctx, "precondition", pre)
        assert kf.kfac_get_status(ctx)[0] == 0
    ref = outputs(ref_st)
    lf = kf.step_descs(layers)
    st = state()
    ea, inv, pre = descs(st)
    F0 = [f.clone() for f in st["F"]]
    stream = torch.cuda.Stream()
    with kf.Context(0, stream) as ctx:
        with torch.cuda.stream(stream):
            kf.kfac_step_grouped(ctx, ea, inv, pre, lf)
            stream.synchronize()
        assert kf.kfac_get_status(ctx)[0] == 0
        got = outputs(st)
        for a, b in zip(ref, got):
            assert torch.equal(a, b)
        for f, f0 in zip(st["F"], F0):
            f.copy_(f0)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            kf.kfac_step_grouped(ctx, ea, inv, pre, lf)
        for f, f0 in zip(st["F"], F0):
            f.copy_(f0)
        with torch.cuda.stream(stream):
            g.replay()
            stream.synchronize()
        assert kf.kfac_get_status(ctx)[0] == 0
        for a, b in zip(ref, outputs(st)):
            assert torch.equal(a, b)
