"""Test-side workload assembly: seeded inputs (from the generator module) turned
into the K-factors the paper's networks produce (Sec. 5 / Sec. 3 recipe).

Factors used as *inputs* to the inversion tests are accumulated in FP64 (the
oracle's EA for small d, a BLAS product for the large, full-size cases) and
rounded to FP32; nothing here comes from the CUDA path."""
import numpy as np

import oracle
from paper_2206_15397_gb300 import inputs


def ea_factor(xs, rho=0.95, use_oracle=True):
    d = xs[0].shape[0]
    f = np.zeros((d, d))
    for x in xs:
        x64 = x.astype(np.float64)
        if use_oracle:
            f = oracle.ea_update(f, x64, rho)
        else:
            f = rho * f + (1.0 - rho) * (x64 @ x64.T) / x64.shape[1]
    return f


def c1(seed=0, g_scale=1e-3):
    """Single factor pair: A 512x512 and G 256x256 from 10 EA steps of n=128
    activations (s_i = i^-1, G scaled 1e-3), J 256x512 ~ N(0, 1e-2), r=64, p=10,
    q=1, lambda=0.1."""
    xa = inputs.activation_batches(seed, 512, 128, 10, alpha=1.0, salt=1)
    xg = inputs.activation_batches(seed, 256, 128, 10, alpha=1.0, scale=g_scale, salt=2)
    fa = ea_factor(xa).astype(np.float32)
    fg = ea_factor(xg).astype(np.float32)
    j = inputs.gradient(seed, 256, 512, std=0.1)
    return dict(fa=fa, fg=fg, j=j, r=64, p=10, q=1, lam=0.1,
                om_a=inputs.omega(seed, 512, 74, salt=1), om_g=inputs.omega(seed, 256, 74, salt=2))


def spectral(seed, d, k, alpha=1.5, n=64, steps=4, bias=False, use_oracle=True, scale=1.0):
    xs = inputs.activation_batches(seed, d - (1 if bias else 0), n, steps, alpha=alpha, scale=scale, bias=bias,
                                   salt=7)
    f = ea_factor(xs, use_oracle=use_oracle).astype(np.float32)
    return f, inputs.omega(seed, d, k, salt=7)
