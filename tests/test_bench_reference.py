"""The CPU leg of bench.py (the reference arm times the FP64 oracle on a
bounded sample of a step and projects it to one step) on a tiny workload, so
that its sampling and projection logic runs in the CPU suite."""
import numpy as np
import pytest


def test_oracle_step_sample_small():
    import bench
    import oracle
    from paper_2206_15397_gb300 import inputs as I
    oracle.build()
    w = dict(bench.WORKLOAD)
    w.update(d_in=63, d_out=64, n=16, r=12, p=4)
    da, dg, k = w["d_in"] + int(w["bias"]), w["d_out"], w["r"] + w["p"]
    xa = I.activation_batches(w["seed"], w["d_in"], w["n"], 1, alpha=w["alpha"], bias=w["bias"], salt=11)[0]
    v = I.haar(w["seed"], dg, salt=12)
    fg = ((v * I.power_spectrum(dg, 2 * w["alpha"])[None, :]) @ v.T).astype(np.float32)
    fa = np.eye(da, dtype=np.float32)
    fa[:dg, :dg] = fg
    j = I.gradient(w["seed"], dg, da, std=w["j_std"], salt=20)
    om = I.omega(w["seed"], dg, k, salt=40)
    for frac in (1, 4):
        ms, spent = bench.oracle_step_sample(w, 1, fa, fg, j, om, xa, frac)
        assert np.isfinite(ms) and ms > 0.0
        assert spent > 0.0
