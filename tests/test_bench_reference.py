"""The CPU legs of bench.py (the reference arm and the CPU baseline time the FP64
oracle on one layer of the step and scale each stage by its work over the whole
step) on a tiny workload, so that their sampling and scaling logic runs in the
CPU suite."""
import numpy as np


def tiny_spec():
    factors = [dict(d=41, alpha=1.0, r=6, bias=True), dict(d=24, alpha=1.5, r=6, bias=False),
               dict(d=12, alpha=1.0, r=10, bias=False), dict(d=30, alpha=1.2, r=4, bias=False)]
    return dict(name="tiny", factors=factors, layers=[(0, 1), (2, 3)], n=8, p=4, q=1, lam=0.1, rho=0.95,
                m_cap=None, seed=0, j_std=0.1, workload="tiny")


def test_oracle_projected_step_tiny():
    import bench
    spec = tiny_spec()
    for li in range(2):
        ms, spent, times = bench.oracle_projected_step(spec, li, 2)
        assert np.isfinite(ms) and ms > 0.0 and spent > 0.0
        assert set(times) == {"ea", "prod", "qr", "proj", "jacobi", "lift", "apply"}
    # layer 1: factor 2 takes the exact path (k = 14 >= d = 12, Jacobi on d x d), factor 3 is sketched (k = 8)
    w = bench.oracle_stage_work(spec, [1])
    assert w["jacobi"] == 12.0 ** 3 + 8.0 ** 3 and w["prod"] == 3.0 * 30 * 30 * 8


def test_pick_layer_and_stage_work():
    import bench
    spec = tiny_spec()
    assert bench.pick_layer(spec, 1, 1e9) in (0, 1)
    assert bench.pick_layer(spec, 1, 0.0) == min(range(2), key=lambda li: sum(bench.oracle_stage_work(spec, [li]).values()))
    f, b = bench.stage_work("sketch_gemm", spec)
    assert f == 3 * 2.0 * 10 * 41 * 41 + 3 * 2.0 * 10 * 24 * 24 + 3 * 2.0 * 8 * 30 * 30 and b > 0


def test_workload_specs():
    import bench
    c5 = bench.workload_spec("c5")
    assert len(c5["factors"]) == 64 and len(c5["layers"]) == 32
    assert all(256 <= f["d"] <= 8192 and f["r"] in (64, 128, 256, 512) or f["r"] == f["d"] for f in c5["factors"])
    c3 = bench.workload_spec("c3")
    assert [f["d"] for f in c3["factors"][::2]] == [28, 577, 577, 1153, 1153, 2305, 2305, 2305, 4609, 4609, 4609,
                                                     4609, 4609, 513]
    assert [f["d"] for f in c3["factors"][1::2]] == [64, 64, 128, 128, 256, 256, 256, 512, 512, 512, 512, 512, 512, 10]
    c2 = bench.workload_spec("c2", q=2)
    assert [f["d"] for f in c2["factors"]] == [4097, 4096] and c2["q"] == 2
