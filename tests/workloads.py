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


# VGG16_bn on 32x32 images (Sec. 5): 13 conv layers (3x3 kernels, A factor
# C_in * 9 + 1 with the bias row, G factor C_out) and the final FC layer
# (512 + 1 -> 10).
C3_CONV = [(3, 64), (64, 64), (64, 128), (128, 128), (128, 256), (256, 256), (256, 256), (256, 512), (512, 512),
           (512, 512), (512, 512), (512, 512), (512, 512)]


def c3(seed=0, n=128, steps=10, alpha=1.0, rank_cap=512, g_scale=1.0):
    """The VGG16_bn factor set: per layer A (C_in*9 + 1) and G (C_out) factors
    from `steps` EA steps of n activations / gradients with s_i = i^-alpha
    (directions beyond rank_cap dropped), J ~ N(0, 1e-2), r = min(d, 220),
    p = 10, q = 1, lambda = 0.1. Factors in FP32, accumulated in FP64."""
    layers = []
    dims = [(ci * 9, co) for ci, co in C3_CONV] + [(512, 10)]
    for li, (din, dout) in enumerate(dims):
        xa = inputs.activation_batches(seed, din, n, steps, alpha=alpha, bias=True, salt=100 + li, rank_cap=rank_cap)
        xg = inputs.activation_batches(seed, dout, n, steps, alpha=alpha, scale=g_scale, salt=200 + li,
                                       rank_cap=rank_cap)
        fa = ea_factor(xa, use_oracle=False).astype(np.float32)
        fg = ea_factor(xg, use_oracle=False).astype(np.float32)
        da, dg = din + 1, dout
        layers.append(dict(fa=fa, fg=fg, j=inputs.gradient(seed, dg, da, std=0.1, salt=300 + li),
                           om_a=inputs.omega(seed, da, min(da, 220) + 10, salt=400 + li),
                           om_g=inputs.omega(seed, dg, min(dg, 220) + 10, salt=500 + li),
                           r_a=min(da, 220), r_g=min(dg, 220)))
    return dict(layers=layers, p=10, q=1, lam=0.1)
