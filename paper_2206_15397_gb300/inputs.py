"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module draws random numbers and shapes them into the workloads' inputs:
activation and gradient batches, gradient matrices, Gaussian test matrices and
factors with a prescribed spectrum. It holds none of the randomized K-FAC
arithmetic (no EA update, no sketch, no orthonormalisation, no eigensolve, no
damping) so that the FP64 oracle and the CUDA path can both be fed from it.

Randomness comes from one counter-based generator written from its published
definition: Philox4x32 with 10 rounds (Salmon, Moraes, Dror and Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), turned into standard normals by
the Box-Muller transform in FP64. A draw is addressed by (seed, stream,
element index), so the same seed gives the same numbers on any machine.

Workload recipe (activations shaped like the paper's networks, Sec. 5, with the
fast spectral decay of Sec. 3): a batch of n activation vectors of a layer with
d inputs is a = z diag(s) V^T with z ~ N(0,1)^{n x d}, s_i = scale * i^-alpha
and V a Haar-distributed orthogonal matrix; the K-factor batch matrix is its
transpose, shape (d, n). Layers with a bias get a row of ones appended last.
"""
from __future__ import annotations

import math

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox4x32-10 block function, vectorised over the leading axis.

    ctr: uint32 array (..., 4); key: uint32 array (..., 2). Each round computes
    the two 32x32->64 products of words 0 and 2 with the round multipliers, mixes
    the high halves with words 1/3 and the key, and bumps the key by the Weyl
    constants."""
    x = [ctr[..., i].astype(np.uint32) for i in range(4)]
    k0 = key[..., 0].astype(np.uint32).copy()
    k1 = key[..., 1].astype(np.uint32).copy()
    with np.errstate(over="ignore"):
        for rnd in range(10):
            p0 = _M0 * x[0].astype(np.uint64)
            p1 = _M1 * x[2].astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            x = [hi1 ^ x[1] ^ k0, lo1, hi0 ^ x[3] ^ k1, lo0]
            if rnd != 9:
                k0 = k0 + _W0
                k1 = k1 + _W1
    return np.stack(x, axis=-1)


def _uniform53(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Two uint32 words -> a double strictly inside (0, 1) with 53 random bits."""
    hi = (a >> np.uint32(5)).astype(np.float64)   # 27 bits
    lo = (b >> np.uint32(6)).astype(np.float64)   # 26 bits
    return (hi * 67108864.0 + lo + 0.5) / 9007199254740992.0


def standard_normal(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """`count` i.i.d. N(0, 1) FP64 values for (seed, stream)."""
    nblk = (count + 1) // 2
    idx = np.arange(nblk, dtype=np.uint64)
    ctr = np.zeros((nblk, 4), dtype=np.uint32)
    ctr[:, 0] = (idx & _MASK32).astype(np.uint32)
    ctr[:, 1] = (idx >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = np.uint32(stream & 0xFFFFFFFF)
    ctr[:, 3] = np.uint32((stream >> 32) & 0xFFFFFFFF)
    key = np.empty((nblk, 2), dtype=np.uint32)
    key[:, 0] = np.uint32(seed & 0xFFFFFFFF)
    key[:, 1] = np.uint32((seed >> 32) & 0xFFFFFFFF)
    w = philox4x32_10(ctr, key)
    u1 = _uniform53(w[:, 0], w[:, 1])
    u2 = _uniform53(w[:, 2], w[:, 3])
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * nblk)
    z[0::2] = rad * np.cos(2.0 * math.pi * u2)
    z[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return z[:count]


def uniform(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """`count` i.i.d. U(0, 1) FP64 values for (seed, stream) (one Philox block each)."""
    idx = np.arange(count, dtype=np.uint64)
    ctr = np.zeros((count, 4), dtype=np.uint32)
    ctr[:, 0] = (idx & _MASK32).astype(np.uint32)
    ctr[:, 1] = (idx >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = np.uint32(stream & 0xFFFFFFFF)
    ctr[:, 3] = np.uint32((stream >> 32) & 0xFFFFFFFF)
    key = np.empty((count, 2), dtype=np.uint32)
    key[:, 0] = np.uint32(seed & 0xFFFFFFFF)
    key[:, 1] = np.uint32((seed >> 32) & 0xFFFFFFFF)
    w = philox4x32_10(ctr, key)
    return _uniform53(w[:, 0], w[:, 1])


# Streams keep the draws of different objects of one workload independent.
STREAM_OMEGA = 1
STREAM_HAAR = 2
STREAM_BATCH = 3
STREAM_GRAD = 4
STREAM_MISC = 5
STREAM_SHAPES = 6


def gaussian(seed: int, shape, stream: int = STREAM_MISC, std: float = 1.0) -> np.ndarray:
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape)) if shape else 1
    return (std * standard_normal(seed, n, stream)).reshape(shape)


def omega(seed: int, d: int, k: int, salt: int = 0) -> np.ndarray:
    """Gaussian test matrix Omega (d x k) of Alg. 3, rounded to FP32 so that the
    oracle and the GPU consume bit-identical values."""
    z = gaussian(seed, (d, k), stream=(STREAM_OMEGA << 32) + salt)
    return z.astype(np.float32)


def seeded_omega(seed: int, d: int, k: int) -> np.ndarray:
    """The d x k Gaussian test matrix the library draws on the device for `seed`
    (its seed path): value e = i*k + j of element (i, j) comes from Philox block
    e // 4 with the counter (block mod 2^32, block // 2^32, 0, 1); a word w maps
    to u = (floor(w / 512) + 1/2) / 2^23 (exact in FP32); words 0, 1 give the Box-Muller pair
    sqrt(-2 ln u0) (cos, sin)(2 pi u1) (values 4b, 4b+1), words 2, 3 the next
    pair. Evaluated here in FP64 and rounded to FP32 (the device evaluates the
    same formula in FP32)."""
    n = int(d) * int(k)
    nblk = (n + 3) // 4
    idx = np.arange(nblk, dtype=np.uint64)
    ctr = np.zeros((nblk, 4), dtype=np.uint32)
    ctr[:, 0] = (idx & _MASK32).astype(np.uint32)
    ctr[:, 1] = (idx >> np.uint64(32)).astype(np.uint32)
    ctr[:, 3] = np.uint32(1)
    key = np.empty((nblk, 2), dtype=np.uint32)
    key[:, 0] = np.uint32(seed & 0xFFFFFFFF)
    key[:, 1] = np.uint32((seed >> 32) & 0xFFFFFFFF)
    w = philox4x32_10(ctr, key)
    u = ((w >> np.uint32(9)).astype(np.float64) + 0.5) / 8388608.0
    z = np.empty((nblk, 4))
    for a in (0, 2):
        rho = np.sqrt(-2.0 * np.log(u[:, a]))
        ang = 2.0 * math.pi * u[:, a + 1]
        z[:, a] = rho * np.cos(ang)
        z[:, a + 1] = rho * np.sin(ang)
    return z.reshape(-1)[:n].reshape(int(d), int(k)).astype(np.float32)


def haar(seed: int, d: int, salt: int = 0) -> np.ndarray:
    """Haar-distributed orthogonal d x d matrix: QR of a Gaussian matrix with the
    signs of diag(R) moved into Q (Mezzadri 2007)."""
    g = gaussian(seed, (d, d), stream=(STREAM_HAAR << 32) + salt)
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))[None, :]


def stiefel(seed: int, d: int, m: int, salt: int = 0) -> np.ndarray:
    """d x m matrix with orthonormal columns, uniformly distributed (the first m
    columns of a Haar matrix): QR of a d x m Gaussian with the signs of diag(R)
    moved into Q."""
    g = gaussian(seed, (d, m), stream=(STREAM_HAAR << 32) + (1 << 24) + salt)
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))[None, :]


def power_spectrum(d: int, alpha: float, scale: float = 1.0) -> np.ndarray:
    i = np.arange(1, d + 1, dtype=np.float64)
    return scale * i ** (-alpha)


def activation_batches(seed: int, d: int, n: int, steps: int, alpha: float, scale: float = 1.0,
                       bias: bool = False, salt: int = 0, v: np.ndarray | None = None,
                       rank_cap: int | None = None):
    """`steps` batch matrices of shape (d_out, n), d_out = d + bias, drawn as
    a = z diag(s) V^T (one row of a per sample) and transposed. Returns FP32.
    With rank_cap = m < d only the m leading directions are drawn (V is d x m,
    uniform on the Stiefel manifold, s = s_1..s_m): the same recipe with the
    spectrum cut off at m, which keeps generation O(d m^2) for wide layers."""
    m = d if rank_cap is None else min(d, int(rank_cap))
    if v is None:
        v = haar(seed, d, salt) if m == d else stiefel(seed, d, m, salt)
    s = power_spectrum(m, alpha, scale)
    vs = v[:, :m] * s[None, :]              # V diag(s)
    out = []
    for t in range(steps):
        z = gaussian(seed, (n, m), stream=(STREAM_BATCH << 32) + (salt << 16) + t)
        x = vs @ z.T                        # (d, n) = V diag(s) z^T
        if bias:
            x = np.vstack([x, np.ones((1, n))])
        out.append(x.astype(np.float32))
    return out


def gradient(seed: int, dg: int, da: int, std: float, salt: int = 0) -> np.ndarray:
    """Gradient matrix J = Mat(g) (d_g x d_a) ~ N(0, std^2), FP32."""
    return gaussian(seed, (dg, da), stream=(STREAM_GRAD << 32) + salt, std=std).astype(np.float32)


def spectrum_factor(seed: int, d: int, spectrum, salt: int = 0) -> np.ndarray:
    """Symmetric d x d matrix V diag(spectrum) V^T with V Haar (FP64)."""
    v = haar(seed, d, salt)
    sp = np.asarray(spectrum, dtype=np.float64)
    return (v * sp[None, :]) @ v.T


def low_rank_factor(seed: int, d: int, spectrum, salt: int = 0):
    """Rank-len(spectrum) PSD matrix V_r diag(s) V_r^T and its exact eigenpairs."""
    sp = np.asarray(spectrum, dtype=np.float64)
    v = haar(seed, d, salt)[:, : sp.shape[0]]
    return (v * sp[None, :]) @ v.T, v, sp


def batching_stress_shapes(seed: int = 0, count: int = 64):
    """The batching-stress factor set: per factor d ~ U{256..8192}, decay
    alpha ~ U[0.8, 2], rank r from {64, 128, 256, 512} capped at d (seeded)."""
    u = uniform(seed, 3 * count, stream=STREAM_SHAPES << 32)
    d = 256 + np.minimum((u[0::3] * (8192 - 256 + 1)).astype(np.int64), 8192 - 256)
    alpha = 0.8 + 1.2 * u[1::3]
    r = np.array([64, 128, 256, 512])[np.minimum((u[2::3] * 4).astype(np.int64), 3)]
    return [dict(d=int(di), alpha=float(ai), r=int(min(ri, di))) for di, ai, ri in zip(d, alpha, r)]
