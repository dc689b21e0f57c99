"""Pins for the FP64 oracle: each test checks it against something other than
itself (the paper's printed values, closed forms, library routines on special
cases, invariants, brute force on tiny inputs)."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2206_15397_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rng(seed):
    return np.random.default_rng(seed)


def rand_sym(n, seed):
    a = rng(seed).standard_normal((n, n))
    return 0.5 * (a + a.T)


def rand_psd(n, seed, rank=None):
    x = rng(seed).standard_normal((n, rank or n))
    return x @ x.T / (rank or n)


# ----------------------------------------------------------------------------- EA update

@pytest.mark.parametrize("d,n,steps,rho", [(1, 1, 1, 0.95), (7, 3, 5, 0.95), (33, 16, 10, 0.9), (20, 40, 4, 0.5)])
def test_ea_matches_closed_form(d, n, steps, rho):
    """Eq. (6): the recursion unrolls to rho^K F0 + (1-rho) sum_i rho^(K-1-i) X_i X_i^T / n."""
    f0 = rand_psd(d, 1)
    xs = [rng(10 + t).standard_normal((d, n)) for t in range(steps)]
    f = f0.copy()
    for x in xs:
        f = oracle.ea_update(f, x, rho)
    closed = rho ** steps * f0
    for i, x in enumerate(xs):
        closed = closed + (1 - rho) * rho ** (steps - 1 - i) * np.einsum("at,bt->ab", x, x) / n
    np.testing.assert_allclose(f, closed, rtol=1e-12, atol=1e-14)


def test_ea_special_cases():
    x = rng(3).standard_normal((9, 5))
    f0 = rand_psd(9, 4)
    # rho = 0: the factor is the batch statistic X X^T / n alone (a library matmul).
    np.testing.assert_allclose(oracle.ea_update(f0, x, 0.0), x @ x.T / 5, rtol=1e-13)
    # rho = 1: the factor does not move.
    np.testing.assert_array_equal(oracle.ea_update(f0, x, 1.0), f0)
    # Identity initialisation of Alg. 1 after K steps: rho^K I + EA sum.
    f = np.eye(9)
    f = oracle.ea_update(f, x, 0.95)
    np.testing.assert_allclose(f, 0.95 * np.eye(9) + 0.05 * x @ x.T / 5, rtol=1e-13)


def test_ea_symmetric_psd():
    f = np.zeros((40, 40))
    for t in range(10):
        f = oracle.ea_update(f, rng(t).standard_normal((40, 8)), 0.95)
    np.testing.assert_array_equal(f, f.T)
    w = np.linalg.eigvalsh(f)
    assert w.min() >= -1e-12 * w.max()
    # rank <= K n (the observation behind Prop. 3.1): 10 steps of 8 columns < 40 is not
    # binding here, so use a thinner case.
    g = np.zeros((40, 40))
    for t in range(3):
        g = oracle.ea_update(g, rng(50 + t).standard_normal((40, 4)), 0.95)
    assert np.linalg.matrix_rank(g, tol=1e-10 * np.abs(g).max()) == 12


# ----------------------------------------------------------------------------- Jacobi

def test_jacobi_2x2_closed_form():
    a, b, c = 2.0, -0.7, 0.5
    w, v, _ = oracle.jacobi_eigh(np.array([[a, b], [b, c]]))
    mid, rad = (a + c) / 2, math.hypot((a - c) / 2, b)
    np.testing.assert_allclose(w, [mid + rad, mid - rad], rtol=1e-15)
    # eigenvector of the larger eigenvalue is proportional to (b, lambda1 - a)
    e = np.array([b, mid + rad - a])
    e /= np.linalg.norm(e)
    assert abs(abs(e @ v[:, 0]) - 1) < 1e-14


def test_jacobi_diagonal_and_order():
    d = np.array([3.0, -1.0, 7.0, 0.0, 3.0])
    w, v, sweeps = oracle.jacobi_eigh(np.diag(d))
    np.testing.assert_array_equal(w, [7.0, 3.0, 3.0, 0.0, -1.0])
    assert sweeps == 0
    # ties keep the original index order: both 3.0 eigenvectors are e_0 then e_4
    np.testing.assert_array_equal(np.abs(v[:, 1]), np.eye(5)[:, 0])
    np.testing.assert_array_equal(np.abs(v[:, 2]), np.eye(5)[:, 4])


@pytest.mark.parametrize("n", [1, 2, 3, 7, 31, 40])
def test_jacobi_vs_library(n):
    a = rand_sym(n, n)
    w, v, sweeps = oracle.jacobi_eigh(a)
    assert sweeps >= 0
    np.testing.assert_allclose(w, np.linalg.eigvalsh(a)[::-1], atol=1e-13 * max(1, np.abs(a).max()))
    assert np.all(np.diff(w) <= 0)
    nrm = np.linalg.norm(a)
    assert np.linalg.norm(a @ v - v * w[None, :]) <= 1e-13 * max(nrm, 1e-300) * n
    np.testing.assert_allclose(v.T @ v, np.eye(n), atol=1e-14 * n)


def _det_bruteforce(a):
    n = a.shape[0]
    tot = 0.0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        prod = 1.0
        for i in range(n):
            prod *= a[i, perm[i]]
        tot += (-1) ** inv * prod
    return tot


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_jacobi_bruteforce_invariants(n):
    """Tiny sizes: each eigenvalue is a root of det(A - lam I) (Leibniz expansion),
    and sum(lam) = trace, prod(lam) = det, sum(lam^2) = ||A||_F^2."""
    a = rand_sym(n, 100 + n)
    w, _, _ = oracle.jacobi_eigh(a)
    scale = np.abs(a).max() ** n
    for lam in w:
        assert abs(_det_bruteforce(a - lam * np.eye(n))) <= 1e-11 * scale
    assert abs(w.sum() - np.trace(a)) <= 1e-13
    assert abs(np.prod(w) - _det_bruteforce(a)) <= 1e-12 * scale
    assert abs((w ** 2).sum() - (a ** 2).sum()) <= 1e-12 * (a ** 2).sum()


def test_jacobi_prescribed_spectrum():
    s = np.array([5.0, 2.0, 2.0, 1e-3, 0.0, 0.0, -0.5])
    a = inputs.spectrum_factor(7, 7, s)
    w, v, _ = oracle.jacobi_eigh(a)
    np.testing.assert_allclose(w, s, atol=1e-14 * 5)


# ----------------------------------------------------------------------------- QR

@pytest.mark.parametrize("m,k", [(1, 1), (5, 5), (9, 3), (64, 17), (130, 40)])
def test_qr_properties_and_library(m, k):
    y = rng(m * k).standard_normal((m, k))
    q, r = oracle.qr(y)
    np.testing.assert_allclose(q.T @ q, np.eye(k), atol=1e-14 * max(1, k))
    np.testing.assert_allclose(q @ r, y, atol=1e-13 * np.abs(y).max())
    assert np.all(np.tril(r, -1) == 0)
    assert np.all(np.diag(r) >= 0)
    # unique for full rank: equals LAPACK's QR once diag(R) is made positive
    ql, rl = np.linalg.qr(y)
    sg = np.sign(np.diag(rl))
    np.testing.assert_allclose(q, ql * sg[None, :], atol=1e-12)
    np.testing.assert_allclose(r, rl * sg[:, None], atol=1e-12 * np.abs(y).max())


def test_qr_rank_deficient():
    y = rng(7).standard_normal((30, 6))
    y[:, 3] = y[:, 1]          # duplicate column
    y[:, 5] = 0.0              # zero column
    q, r = oracle.qr(y)
    np.testing.assert_allclose(q.T @ q, np.eye(6), atol=1e-13)
    np.testing.assert_allclose(q @ r, y, atol=1e-13)


# ----------------------------------------------------------------------------- SREVD

def test_srevd_exact_recovery_low_rank():
    """rank(X) <= r: the sketch captures range(X) exactly, so there is no
    projection error (Sec. 2.2.1) and the r modes are recovered exactly."""
    d, r, p = 60, 6, 4
    s = np.array([4.0, 2.0, 1.0, 0.5, 0.2, 0.1])
    x, v, _ = inputs.low_rank_factor(3, d, s)
    om = inputs.omega(3, d, r + p).astype(np.float64)
    for q in (0, 1, 2):
        u, dd = oracle.srevd(x, om, q, r)
        np.testing.assert_allclose(dd, s, rtol=1e-12)
        np.testing.assert_allclose(u @ np.diag(dd) @ u.T, x, atol=1e-12)
        np.testing.assert_allclose(u @ u.T, v @ v.T, atol=1e-12)


def test_srevd_k_ge_d_is_full_evd():
    d = 12
    x = rand_psd(d, 5)
    om = inputs.omega(5, d, 14).astype(np.float64)
    u, dd = oracle.srevd(x, om, 1, 20)
    assert u.shape == (d, d)
    np.testing.assert_allclose(dd, np.linalg.eigvalsh(x)[::-1], atol=1e-14)
    np.testing.assert_allclose(u @ np.diag(dd) @ u.T, x, atol=1e-13)


def test_srevd_ritz_values_interlace_and_basis():
    """Rayleigh-Ritz on any k-dimensional subspace gives theta_i <= lambda_i
    (Cauchy interlacing); C is Q^T X Q of an orthonormal Q."""
    d, k = 80, 12
    x = inputs.spectrum_factor(9, d, inputs.power_spectrum(d, 1.0))
    om = inputs.omega(9, d, k).astype(np.float64)
    u, dd, qb, cb = oracle.srevd(x, om, 0, k, return_basis=True)
    lam = np.linalg.eigvalsh(x)[::-1]
    assert np.all(dd <= lam[:k] + 1e-13)
    np.testing.assert_allclose(qb.T @ qb, np.eye(k), atol=1e-13)
    np.testing.assert_allclose(cb, qb.T @ x @ qb, atol=1e-13)
    np.testing.assert_allclose(u.T @ u, np.eye(k), atol=1e-13)
    # Ritz pairs: U^T X U = diag(D)
    np.testing.assert_allclose(u.T @ x @ u, np.diag(dd), atol=1e-13)


def test_range_finder_halko_bound():
    """Expected-error bound of the Gaussian range finder (Halko, Martinsson and
    Tropp 2011, Thm. 10.5): E||X - QQ^T X||_F <= (1 + r/(p-1))^(1/2) (sum_{j>r} s_j^2)^(1/2)."""
    d, r, p = 70, 8, 5
    sv = inputs.power_spectrum(d, 1.0)
    x = inputs.spectrum_factor(11, d, sv)
    errs = []
    for seed in range(50):
        om = inputs.omega(seed, d, r + p).astype(np.float64)
        _, _, qb, _ = oracle.srevd(x, om, 0, r, return_basis=True)
        errs.append(np.linalg.norm(x - qb @ (qb.T @ x)))
    bound = math.sqrt(1 + r / (p - 1)) * math.sqrt((sv[r:] ** 2).sum())
    assert np.mean(errs) <= bound
    # and the error is never below the optimal rank-(r+p) truncation error
    assert min(errs) >= math.sqrt((sv[r + p:] ** 2).sum()) * (1 - 1e-12)


def test_power_iterations_reduce_error():
    d, r, p = 90, 10, 3
    sv = inputs.power_spectrum(d, 0.5)
    x = inputs.spectrum_factor(12, d, sv)
    best = np.sqrt((sv[r:] ** 2).sum())
    mean_err = []
    for q in (0, 1, 2):
        e = []
        for seed in range(20):
            om = inputs.omega(seed, d, r + p).astype(np.float64)
            u, dd = oracle.srevd(x, om, q, r)
            e.append(np.linalg.norm(x - u @ np.diag(dd) @ u.T))
        mean_err.append(np.mean(e))
    assert mean_err[0] > mean_err[1] > mean_err[2] >= best * (1 - 1e-12)


# ----------------------------------------------------------------------------- damping / apply

def test_damped_coef_values():
    c = oracle.damped_coef(np.array([0.1, 0.0, -1e-9, 1.0]), 0.1)
    np.testing.assert_allclose(c, [1 / 0.2 - 10, 0.0, 0.0, 1 / 1.1 - 10], rtol=1e-15)


def test_eq13_lowrank_inverse_vs_solve():
    """Eq. (13) against a direct dense solve of (U D U^T + lam I) S = V."""
    d, r, lam = 15, 4, 0.3
    u, _ = np.linalg.qr(rng(1).standard_normal((d, r)))
    dv = np.array([3.0, 1.0, 0.2, 0.01])
    vmat = rng(2).standard_normal((d, 6))
    c = oracle.damped_coef(dv, lam)
    lhs = u @ (c[:, None] * (u.T @ vmat)) + vmat / lam
    direct = np.linalg.solve(u @ np.diag(dv) @ u.T + lam * np.eye(d), vmat)
    np.testing.assert_allclose(lhs, direct, rtol=1e-12, atol=1e-12)


def _inv(a):
    return np.linalg.inv(a)


def test_precondition_full_rank_equals_exact_inverse():
    """With r = d, Alg. 4's M/S updates equal (G + lam I)^-1 J (A + lam I)^-1 (Sec. 2.1)."""
    da, dg, lam = 9, 6, 0.05
    fa, fg = rand_psd(da, 1), rand_psd(dg, 2)
    j = rng(3).standard_normal((dg, da))
    wa, va, _ = oracle.jacobi_eigh(fa)
    wg, vg, _ = oracle.jacobi_eigh(fg)
    s = oracle.precondition(j, va, oracle.damped_coef(wa, lam), vg, oracle.damped_coef(wg, lam), lam)
    ref = np.linalg.solve(fg + lam * np.eye(dg), j) @ _inv(fa + lam * np.eye(da))
    np.testing.assert_allclose(s, ref, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(oracle.exact_apply(j, fa, fg, lam), ref, rtol=1e-10, atol=1e-10)


def test_precondition_rank_one_closed_form():
    """J = u v^T with u, v eigenvectors of G, A: S = u v^T / ((lam_u + lam)(lam_v + lam))."""
    da, dg, lam = 8, 5, 0.2
    fa = inputs.spectrum_factor(1, da, np.linspace(2, 0.1, da))
    fg = inputs.spectrum_factor(2, dg, np.linspace(3, 0.5, dg))
    wa, va, _ = oracle.jacobi_eigh(fa)
    wg, vg, _ = oracle.jacobi_eigh(fg)
    iu, iv = 1, 2
    j = np.outer(vg[:, iu], va[:, iv])
    ra, rg = 3, 2   # truncated: v is inside the kept A modes, u inside the kept G modes
    s = oracle.precondition(j, va[:, :ra], oracle.damped_coef(wa[:ra], lam),
                            vg[:, :rg], oracle.damped_coef(wg[:rg], lam), lam)
    np.testing.assert_allclose(s, j / ((wg[iu] + lam) * (wa[iv] + lam)), atol=1e-13)
    # a mode outside the kept set is damped by 1/lam only
    j2 = np.outer(vg[:, 4], va[:, 6])
    s2 = oracle.precondition(j2, va[:, :ra], oracle.damped_coef(wa[:ra], lam),
                             vg[:, :rg], oracle.damped_coef(wg[:rg], lam), lam)
    np.testing.assert_allclose(s2, j2 / lam ** 2, atol=1e-13)


def test_precondition_cols_full_rank_equals_exact_inverse():
    """Selected columns with r = d equal the columns of (G + lam I)^-1 J (A + lam I)^-1."""
    da, dg, lam = 11, 7, 0.05
    fa, fg = rand_psd(da, 4), rand_psd(dg, 5)
    j = rng(6).standard_normal((dg, da))
    wa, va, _ = oracle.jacobi_eigh(fa)
    wg, vg, _ = oracle.jacobi_eigh(fg)
    cols = np.array([0, 3, 10, 3])
    got = oracle.precondition_cols(j, va, oracle.damped_coef(wa, lam), vg, oracle.damped_coef(wg, lam), lam, cols)
    ref = np.linalg.solve(fg + lam * np.eye(dg), j) @ _inv(fa + lam * np.eye(da))
    np.testing.assert_allclose(got, ref[:, cols], rtol=1e-10, atol=1e-10)


def test_precondition_cols_rank_one_closed_form():
    """J = u v^T with v a kept A mode: only column pattern v survives, scaled per Eq. (13)."""
    da, dg, lam = 8, 5, 0.2
    fa = inputs.spectrum_factor(1, da, np.linspace(2, 0.1, da))
    fg = inputs.spectrum_factor(2, dg, np.linspace(3, 0.5, dg))
    wa, va, _ = oracle.jacobi_eigh(fa)
    wg, vg, _ = oracle.jacobi_eigh(fg)
    j = np.outer(vg[:, 1], va[:, 2])
    cols = np.arange(da)
    got = oracle.precondition_cols(j, va[:, :3], oracle.damped_coef(wa[:3], lam), vg[:, :2],
                                   oracle.damped_coef(wg[:2], lam), lam, cols)
    np.testing.assert_allclose(got, j / ((wg[1] + lam) * (wa[2] + lam)), atol=1e-13)


def test_precondition_empty_ranks():
    j = rng(5).standard_normal((4, 3))
    s = oracle.precondition(j, np.zeros((3, 0)), np.zeros(0), np.zeros((4, 0)), np.zeros(0), 0.5)
    np.testing.assert_allclose(s, j / 0.25, rtol=1e-15)


# ----------------------------------------------------------------------------- Prop. 3.1

def test_prop31_printed_values():
    with open(os.path.join(GOLDEN, "prop31.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert rows
    for eps, alpha, rho, nm, dm, expected in rows:
        assert oracle.rank_bound(float(eps), float(alpha), float(rho), int(nm), int(dm)) == int(expected)
    assert oracle.rank_bound(0.03, 0.1, 0.95, 256, 4097) == 4097  # capped at d_M


def test_prop31_bound_holds_on_ea_factor():
    """On an EA factor built from batches with sigma_max <= sigma_M, the count of
    eigenvalues above eps * lambda_M never exceeds the bound."""
    d, n, rho, steps = 60, 2, 0.5, 40
    f = np.zeros((d, d))
    sig = 0.0
    for t in range(steps):
        x = rng(200 + t).standard_normal((d, n))
        sig = max(sig, np.linalg.norm(x, 2) / math.sqrt(n))
        f = oracle.ea_update(f, x, rho)
    lam = np.linalg.eigvalsh(f)
    alpha = lam.max() / sig ** 2
    eps = 0.05
    count = int((lam >= eps * lam.max()).sum())
    assert count <= oracle.rank_bound(eps, alpha, rho, n, d)


def test_qr_near_identity_stability():
    """Columns almost parallel to e_j: the reflector must be built without
    cancellation (sign of alpha opposite to x_0) to keep Q orthonormal."""
    m, k = 40, 8
    y = np.eye(m, k) + 1e-9 * rng(8).standard_normal((m, k))
    q, r = oracle.qr(y)
    np.testing.assert_allclose(q.T @ q, np.eye(k), atol=1e-14)
    np.testing.assert_allclose(q @ r, y, atol=1e-15)


# ----------------------------------------------------------------------------- one-sided Jacobi SVD (Alg. 2)

@pytest.mark.parametrize("m,n", [(1, 1), (2, 2), (9, 4), (40, 17), (120, 60)])
def test_svd_jacobi_vs_library(m, n):
    """Singular values against LAPACK, the reconstruction U diag(s) V^T = A,
    orthonormal U and V, and each singular triple A v_j = s_j u_j."""
    a = rng(m * 100 + n).standard_normal((m, n))
    u, s, v, sweeps = oracle.svd_jacobi(a)
    assert sweeps > 0
    np.testing.assert_allclose(s, np.linalg.svd(a, compute_uv=False), rtol=1e-12, atol=1e-13)
    assert np.all(np.diff(s) <= 0)
    np.testing.assert_allclose((u * s) @ v.T, a, atol=1e-12)
    np.testing.assert_allclose(u.T @ u, np.eye(n), atol=1e-12)
    np.testing.assert_allclose(v.T @ v, np.eye(n), atol=1e-12)
    np.testing.assert_allclose(a @ v, u * s, atol=1e-12)


def test_svd_jacobi_prescribed_and_degenerate():
    """A = U0 diag(s0) V0^T with Haar factors gives back s0 (distinct values)
    and the right singular subspaces; a zero column gives a zero singular value
    and a zero left vector, without breaking the others."""
    s0 = np.array([5.0, 2.0, 1.0, 0.5, 1e-3])
    u0 = inputs.haar(3, 30)[:, :5]
    v0 = inputs.haar(4, 5)
    u, s, v, _ = oracle.svd_jacobi((u0 * s0) @ v0.T)
    np.testing.assert_allclose(s, s0, rtol=1e-12)
    np.testing.assert_allclose(np.abs(v.T @ v0), np.eye(5), atol=1e-10)   # same vectors up to sign
    a = rng(5).standard_normal((12, 4))
    a[:, 2] = 0.0
    u, s, v, _ = oracle.svd_jacobi(a)
    assert s[-1] == 0.0 and np.all(u[:, -1] == 0.0)
    np.testing.assert_allclose(s[:3], np.linalg.svd(a, compute_uv=False)[:3], rtol=1e-12)


# ----------------------------------------------------------------------------- RSVD (Alg. 2, RS-KFAC)

def test_rsvd_exact_recovery_low_rank():
    """rank(X) <= r: the singular values, the V~ subspace and the rank-r
    reconstruction V~ S~ V~^T are exact (no truncation and no projection error)."""
    s_true = np.array([4.0, 2.0, 1.0, 0.3, 0.05])
    x, v_true, _ = inputs.low_rank_factor(21, 90, s_true)
    om = inputs.gaussian(21, (90, 9))
    v, s = oracle.rsvd(x, om, 0, 5)
    np.testing.assert_allclose(s, s_true, rtol=1e-12)
    np.testing.assert_allclose(v @ v.T, v_true @ v_true.T, atol=1e-12)
    np.testing.assert_allclose((v * s) @ v.T, x, atol=1e-12)


def test_rsvd_singular_values_match_library_svd_of_b():
    """S~ are the leading singular values of B = Q^T X for the basis Q the
    oracle's own QR gives (LAPACK SVD of that B), and with k >= d the RSVD is
    the full eigendecomposition of the PSD factor."""
    x = rand_psd(60, 22, rank=40)
    om = inputs.gaussian(22, (60, 14))
    q, _ = oracle.qr(oracle.matmul(x, om))
    q, _ = oracle.qr(oracle.matmul(x, q))
    b = q.T @ x
    _, s = oracle.rsvd(x, om, 1, 10)
    np.testing.assert_allclose(s, np.linalg.svd(b, compute_uv=False)[:10], rtol=1e-11)
    v, s = oracle.rsvd(x[:12, :12], inputs.gaussian(22, (12, 14)), 1, 12)
    w = np.linalg.eigvalsh(x[:12, :12])[::-1]
    np.testing.assert_allclose(s, w, rtol=1e-11, atol=1e-13)


def test_rsvd_v_is_more_accurate_than_u_and_srevd():
    """Sec. 2.3: V~ approximates the leading eigenvectors better than U~ = Q U_B
    and better than SREVD's Q P_C (mean subspace error over seeds, decaying
    spectrum, no power iteration so the difference is not hidden)."""
    d, r, p = 120, 8, 4
    spec = np.arange(1, d + 1, dtype=float) ** -1.0
    x, v_all, _ = inputs.low_rank_factor(23, d, spec)
    vr = v_all[:, :r]
    err_v, err_u, err_sre = [], [], []
    for seed in range(12):
        om = inputs.gaussian(100 + seed, (d, r + p))
        v, s, u = oracle.rsvd(x, om, 0, r, return_u=True)
        us, _ = oracle.srevd(x, om, 0, r)
        proj = lambda m: np.linalg.norm(m @ m.T - vr @ vr.T)
        err_v.append(proj(v)); err_u.append(proj(u)); err_sre.append(proj(us))
    assert np.mean(err_v) < 0.8 * np.mean(err_u)
    assert np.mean(err_v) < 0.8 * np.mean(err_sre)


def test_rsvd_truncation_dominates_projection_error():
    """Sec. 2.3.1: with V~ the reconstruction error ||X - V~ S~ V~^T||_F is close
    to the truncation error of the exact rank-r eigendecomposition (the
    projection error is small), for a fast-decaying spectrum."""
    d, r = 100, 10
    spec = np.arange(1, d + 1, dtype=float) ** -2.0
    x, _, _ = inputs.low_rank_factor(24, d, spec)
    trunc = np.sqrt(np.sum(spec[r:] ** 2))
    v, s = oracle.rsvd(x, inputs.gaussian(24, (d, r + 10)), 1, r)
    err = np.linalg.norm(x - (v * s) @ v.T)
    assert trunc <= err <= 1.05 * trunc


# ----------------------------------------------------------------------------- conv K-factors (patch statistics)

def _unfold(x, kh, kw, sh, sw, ph, pw):
    """Patch matrix (d x n*ho*wo) by numpy slicing of the zero-padded input."""
    n, c, h, w = x.shape
    xp = np.zeros((n, c, h + 2 * ph, w + 2 * pw))
    xp[:, :, ph:ph + h, pw:pw + w] = x
    ho, wo = (h + 2 * ph - kh) // sh + 1, (w + 2 * pw - kw) // sw + 1
    cols = np.empty((c, kh, kw, n, ho, wo))
    for r in range(kh):
        for t in range(kw):
            cols[:, r, t] = xp[:, :, r:r + sh * ho:sh, t:t + sw * wo:sw].transpose(1, 0, 2, 3)
    return cols.reshape(c * kh * kw, n * ho * wo)


@pytest.mark.parametrize("shape,kernel,stride,pad", [((2, 3, 5, 6), (3, 3), (1, 1), (1, 1)),
                                                      ((3, 2, 7, 7), (3, 2), (2, 1), (0, 1)),
                                                      ((1, 4, 4, 4), (1, 1), (1, 1), (0, 0))])
def test_ea_conv_matches_unfolded_product(shape, kernel, stride, pad):
    """Patch statistics equal the EA update of the explicitly unfolded patch
    matrix (numpy slicing of the zero-padded input), with the bias row."""
    x = rng(sum(shape)).standard_normal(shape)
    a = _unfold(x, *kernel, *stride, *pad)
    abar = np.vstack([a, np.ones((1, a.shape[1]))])
    f0 = rand_psd(abar.shape[0], 3)
    got = oracle.ea_update_conv(f0, x, kernel, stride, pad, 0.9, append_one=True)
    want = 0.9 * f0 + 0.1 * abar @ abar.T / a.shape[1]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13)


def test_ea_conv_special_cases():
    """A kernel covering the whole unpadded image gives one patch per sample
    (the FC factor of the flattened images); a 1 x 1 kernel gives the
    per-position channel covariance; a scale s multiplies the increment by s^2."""
    x = rng(4).standard_normal((5, 2, 3, 4))
    flat = x.reshape(5, -1).T
    got = oracle.ea_update_conv(np.zeros((24, 24)), x, (3, 4), rho=0.5)
    np.testing.assert_allclose(got, oracle.ea_update(np.zeros((24, 24)), flat, 0.5), rtol=1e-12)
    got = oracle.ea_update_conv(np.zeros((2, 2)), x, (1, 1), rho=0.0)
    chan = x.transpose(1, 0, 2, 3).reshape(2, -1)
    np.testing.assert_allclose(got, chan @ chan.T / chan.shape[1], rtol=1e-12)
    g3 = oracle.ea_update_conv(np.zeros((2, 2)), x, (1, 1), rho=0.0, scale=3.0)
    np.testing.assert_allclose(g3, 9.0 * got, rtol=1e-12)
