/*
 * FP64 CPU oracle for the randomized K-FAC hot path (Puiu, "Randomized K-FACs",
 * arXiv 2206.15397).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load or call this library; the product path
 * (the CUDA library) never does, and the two share no code.
 *
 * Everything here is plain, slow FP64 C: triple-loop products, textbook
 * cyclic Jacobi, textbook Householder QR. Each function cites the passage of
 * the paper whose computation it writes out. Matrices are dense, row-major,
 * with the leading dimension equal to the column count. Loops over
 * independent rows or columns carry OpenMP pragmas (used when built with
 * -fopenmp): every output element is still summed by one thread in the same
 * order, so the results are bitwise those of the sequential build.
 *
 * Readings of points where the paper is silent or ambiguous (all mirrored by
 * the GPU path):
 *  - EA normalisation: the batch product A A^T is divided by the column count
 *    n of the batch matrix (Alg. 1 writes A A^T without a 1/n).
 *  - One power iteration = one more product Y <- X Q followed by a fresh
 *    orthonormalisation (Sec. 2.2 mentions power iterations without drawing
 *    them in Alg. 2/3), so the basis spans X^(q+1) Omega.
 *  - Alg. 3 keeps the r leading eigenpairs of C = Q^T X Q, by eigenvalue.
 *  - When k = r + p >= d, there is nothing to sketch: the factor itself is
 *    diagonalised (Q = I) and r is capped at d.
 *  - Negative Ritz values (round-off) are clamped to 0 before damping.
 *
 * Parity status: every function below is pinned by tests that do not re-type
 * its formula (closed forms, library routines on special cases, printed values,
 * invariants). No function is "parity unpinned".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Plain products (a library-free matmul used as a step by the functions     */
/* below).                                                                   */
/* ------------------------------------------------------------------------ */

/* C (m x n) = op(A) op(B), op(A) is m x kk, op(B) is kk x n.
 * ta != 0: A is stored kk x m and op(A) = A^T. tb != 0: B is stored n x kk. */
void orc_matmul(int m, int n, int kk, const double* A, int ta, const double* B, int tb, double* C) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) C[(size_t)i * n + j] = 0.0;
#pragma omp parallel for schedule(dynamic, 8) if ((double)m * n * kk > 1e6)
  for (int i = 0; i < m; ++i) {
    double* c = C + (size_t)i * n;
    for (int t = 0; t < kk; ++t) {
      double a = ta ? A[(size_t)t * m + i] : A[(size_t)i * kk + t];
      if (a == 0.0) continue;
      if (!tb) {
        const double* b = B + (size_t)t * n;
        for (int j = 0; j < n; ++j) c[j] += a * b[j];
      } else {
        for (int j = 0; j < n; ++j) c[j] += a * B[(size_t)j * kk + t];
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* EA K-factor update: Alg. 1, the EA updates of the forward and backward    */
/* factors.                                                                  */
/* (Sec. 2.1), closed form Eq. (6).                                          */
/* ------------------------------------------------------------------------ */

/* F <- rho F + (1 - rho) (1/n) X X^T, X is d x n (one column per sample). */
void orc_ea_update(int d, int n, const double* X, double rho, double* F) {
#pragma omp parallel for schedule(dynamic, 8) if ((double)d * d * n > 1e6)
  for (int i = 0; i < d; ++i) {
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int t = 0; t < n; ++t) s += X[(size_t)i * n + t] * X[(size_t)j * n + t];
      F[(size_t)i * d + j] = rho * F[(size_t)i * d + j] + (1.0 - rho) * s / (double)n;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* EA update of a convolutional layer's K-factor from patch statistics: the  */
/* factor A A^T of Eq. (4) for a conv layer (the paper defers its exact form */
/* to KFC, Sec. 2.1), with A's columns the input patches at every sample and */
/* output position. Reading: the batch product is the mean over samples and  */
/* positions, patches are zero-padded, entries ordered (channel, kernel row, */
/* kernel column) as a conv weight flattens, with the homogeneous 1 last.    */
/* ------------------------------------------------------------------------ */

/* x: n x c x h x w (NCHW). Patch of sample i at output position (oy, ox):
 * p[(ch * kh + r) * kw + t] = x[i, ch, oy * sh + r - ph, ox * sw + t - pw]
 * (0 outside the image), followed by 1 when append_one. Each patch is scaled
 * by `scale`, and F <- rho F + (1 - rho) / (n * ho * wo) * sum_patches p p^T. */
void orc_ea_update_conv(int n, int c, int h, int w, const double* x, int kh, int kw, int sh, int sw, int ph,
                        int pw, int append_one, double scale, double rho, double* F) {
  const int ho = (h + 2 * ph - kh) / sh + 1, wo = (w + 2 * pw - kw) / sw + 1;
  const int d = c * kh * kw + (append_one ? 1 : 0);
  double* S = (double*)calloc((size_t)d * d, sizeof(double));
  double* p = (double*)malloc(sizeof(double) * (size_t)d);
  for (int i = 0; i < n; ++i)
    for (int oy = 0; oy < ho; ++oy)
      for (int ox = 0; ox < wo; ++ox) {
        for (int ch = 0; ch < c; ++ch)
          for (int r = 0; r < kh; ++r)
            for (int t = 0; t < kw; ++t) {
              const int y = oy * sh + r - ph, xx = ox * sw + t - pw;
              const int idx = (ch * kh + r) * kw + t;
              p[idx] = (y >= 0 && y < h && xx >= 0 && xx < w)
                           ? scale * x[(((size_t)i * c + ch) * h + y) * w + xx] : 0.0;
            }
        if (append_one) p[d - 1] = scale;
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b) S[(size_t)a * d + b] += p[a] * p[b];
      }
  const double m = (double)n * ho * wo;
  for (size_t e = 0; e < (size_t)d * d; ++e) F[e] = rho * F[e] + (1.0 - rho) * S[e] / m;
  free(S); free(p);
}

/* ------------------------------------------------------------------------ */
/* Symmetric eigendecomposition by the cyclic-by-row Jacobi method: the      */
/* "eig" of Alg. 1 and the "Eigen_decomp" of Alg. 3.                         */
/* ------------------------------------------------------------------------ */

static void sort_desc(int n, double* w, double* V) {
  /* Stable selection by value, descending; ties keep the original order. */
  int* idx = (int*)malloc(sizeof(int) * (size_t)n);
  double* wt = (double*)malloc(sizeof(double) * (size_t)n);
  double* Vt = (double*)malloc(sizeof(double) * (size_t)n * n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 1; i < n; ++i) { /* insertion sort: stable */
    int v = idx[i], j = i - 1;
    while (j >= 0 && w[idx[j]] < w[v]) { idx[j + 1] = idx[j]; --j; }
    idx[j + 1] = v;
  }
  for (int j = 0; j < n; ++j) {
    wt[j] = w[idx[j]];
    for (int i = 0; i < n; ++i) Vt[(size_t)i * n + j] = V[(size_t)i * n + idx[j]];
  }
  memcpy(w, wt, sizeof(double) * (size_t)n);
  memcpy(V, Vt, sizeof(double) * (size_t)n * n);
  free(idx); free(wt); free(Vt);
}

/* A (n x n symmetric) = V diag(w) V^T. Eigenvalues descending in w, the
 * matching eigenvectors in the columns of V. Sweeps stop once the
 * off-diagonal Frobenius norm is <= tol * ||A||_F, or after max_sweeps.
 * Returns the number of sweeps performed, or -1 if not converged. */
int orc_jacobi_eigh(int n, const double* A_in, double* w, double* V, int max_sweeps, double tol) {
  double* A = (double*)malloc(sizeof(double) * (size_t)n * n);
  memcpy(A, A_in, sizeof(double) * (size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
  double fro = 0.0;
  for (size_t i = 0; i < (size_t)n * n; ++i) fro += A[i] * A[i];
  fro = sqrt(fro);
  int sweeps = 0, converged = 0;
  for (;;) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q)
        if (p != q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
    off = sqrt(off);
    if (off <= tol * fro) { converged = 1; break; }
    if (sweeps >= max_sweeps) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        /* 2x2 symmetric Schur decomposition: the rotation J = [[c, s], [-s, c]]
         * in the (p, q) plane makes (J^T A J)_pq = 0. */
        double tau = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) { /* A <- A J */
          double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) { /* A <- J^T A */
          double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) { /* V <- V J */
          double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
    }
    ++sweeps;
  }
  for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
  free(A);
  sort_desc(n, w, V);
  return converged ? sweeps : -1;
}

/* ------------------------------------------------------------------------ */
/* Thin QR by Householder reflections: the "QR_decomp" of Alg. 2 and Alg. 3. */
/* ------------------------------------------------------------------------ */

/* Y (m x k, m >= k) = Q R, Q m x k with orthonormal columns, R k x k upper
 * triangular with a non-negative diagonal (unique for full-rank Y). */
void orc_qr(int m, int k, const double* Y, double* Q, double* R) {
  double* W = (double*)malloc(sizeof(double) * (size_t)m * k);
  double* Vh = (double*)calloc((size_t)m * k, sizeof(double)); /* Householder vectors */
  double* beta = (double*)calloc((size_t)k, sizeof(double));
  memcpy(W, Y, sizeof(double) * (size_t)m * k);
  for (int j = 0; j < k; ++j) {
    double nrm = 0.0;
    for (int i = j; i < m; ++i) nrm += W[(size_t)i * k + j] * W[(size_t)i * k + j];
    nrm = sqrt(nrm);
    if (nrm == 0.0) { beta[j] = 0.0; continue; }
    double x0 = W[(size_t)j * k + j];
    double alpha = (x0 >= 0.0) ? -nrm : nrm; /* reflect x onto alpha e_1 */
    double vnorm2 = 0.0;
    for (int i = j; i < m; ++i) {
      double v = W[(size_t)i * k + j] - (i == j ? alpha : 0.0);
      Vh[(size_t)i * k + j] = v;
      vnorm2 += v * v;
    }
    if (vnorm2 == 0.0) { beta[j] = 0.0; continue; }
    beta[j] = 2.0 / vnorm2;
#pragma omp parallel for schedule(static) if ((double)(m - j) * (k - j) > 1e5)
    for (int c = j; c < k; ++c) { /* W[j:, c] <- (I - beta v v^T) W[j:, c] */
      double s = 0.0;
      for (int i = j; i < m; ++i) s += Vh[(size_t)i * k + j] * W[(size_t)i * k + c];
      s *= beta[j];
      for (int i = j; i < m; ++i) W[(size_t)i * k + c] -= s * Vh[(size_t)i * k + j];
    }
  }
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) R[(size_t)i * k + j] = (j >= i) ? W[(size_t)i * k + j] : 0.0;
  /* Q = H_0 H_1 ... H_{k-1} [I_k; 0], applied right to left. */
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < k; ++j) Q[(size_t)i * k + j] = (i == j) ? 1.0 : 0.0;
  for (int j = k - 1; j >= 0; --j) {
    if (beta[j] == 0.0) continue;
#pragma omp parallel for schedule(static) if ((double)(m - j) * k > 1e5)
    for (int c = 0; c < k; ++c) {
      double s = 0.0;
      for (int i = j; i < m; ++i) s += Vh[(size_t)i * k + j] * Q[(size_t)i * k + c];
      s *= beta[j];
      for (int i = j; i < m; ++i) Q[(size_t)i * k + c] -= s * Vh[(size_t)i * k + j];
    }
  }
  for (int j = 0; j < k; ++j) { /* make diag(R) non-negative */
    if (R[(size_t)j * k + j] < 0.0) {
      for (int c = 0; c < k; ++c) R[(size_t)j * k + c] = -R[(size_t)j * k + c];
      for (int i = 0; i < m; ++i) Q[(size_t)i * k + j] = -Q[(size_t)i * k + j];
    }
  }
  free(W); free(Vh); free(beta);
}

/* ------------------------------------------------------------------------ */
/* Symmetric randomized EVD with power iterations: Alg. 3 (SREVD), with the  */
/* power iteration of Sec. 2.2.                                              */
/* ------------------------------------------------------------------------ */

/* X: d x d symmetric PSD factor. Omega: d x k Gaussian test matrix (k = r+p).
 * q: power iterations. Outputs: U (d x r_eff), D (r_eff) descending, and
 * optionally the basis Q (d x k) and the projected matrix C (k x k).
 * Returns r_eff = min(r, d), or -1 if a Jacobi solve did not converge. */
int orc_srevd(int d, const double* X, int k, const double* Omega, int q, int r,
              double* U, double* D, double* Q_out, double* C_out) {
  if (r > d) r = d;
  if (k >= d) { /* nothing to sketch: diagonalise the factor itself (Q = I) */
    double* w = (double*)malloc(sizeof(double) * (size_t)d);
    double* V = (double*)malloc(sizeof(double) * (size_t)d * d);
    int rc = orc_jacobi_eigh(d, X, w, V, 100, 1e-15);
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < r; ++j) U[(size_t)i * r + j] = V[(size_t)i * d + j];
    for (int j = 0; j < r; ++j) D[j] = w[j];
    free(w); free(V);
    return rc < 0 ? -1 : r;
  }
  double* Y = (double*)malloc(sizeof(double) * (size_t)d * k);
  double* Q = (double*)malloc(sizeof(double) * (size_t)d * k);
  double* R = (double*)malloc(sizeof(double) * (size_t)k * k);
  double* C = (double*)malloc(sizeof(double) * (size_t)k * k);
  double* w = (double*)malloc(sizeof(double) * (size_t)k);
  double* P = (double*)malloc(sizeof(double) * (size_t)k * k);
  orc_matmul(d, k, d, X, 0, Omega, 0, Y);           /* Y = X Omega        */
  orc_qr(d, k, Y, Q, R);                            /* Q R = QR_decomp(Y) */
  for (int it = 0; it < q; ++it) {                  /* power iterations   */
    orc_matmul(d, k, d, X, 0, Q, 0, Y);             /* Y = X Q            */
    orc_qr(d, k, Y, Q, R);
  }
  orc_matmul(d, k, d, X, 0, Q, 0, Y);               /* Y = X Q            */
  orc_matmul(k, k, d, Q, 1, Y, 0, C);               /* C = Q^T X Q        */
  for (int i = 0; i < k; ++i)                       /* symmetrise         */
    for (int j = i + 1; j < k; ++j) {
      double s = 0.5 * (C[(size_t)i * k + j] + C[(size_t)j * k + i]);
      C[(size_t)i * k + j] = s;
      C[(size_t)j * k + i] = s;
    }
  int rc = orc_jacobi_eigh(k, C, w, P, 100, 1e-15); /* P_C D_C P_C^T = C  */
#pragma omp parallel for schedule(static) if ((double)d * r * k > 1e6)
  for (int i = 0; i < d; ++i)                       /* U = Q P_C[:, :r]   */
    for (int j = 0; j < r; ++j) {
      double s = 0.0;
      for (int t = 0; t < k; ++t) s += Q[(size_t)i * k + t] * P[(size_t)t * k + j];
      U[(size_t)i * r + j] = s;
    }
  for (int j = 0; j < r; ++j) D[j] = w[j];
  if (Q_out) memcpy(Q_out, Q, sizeof(double) * (size_t)d * k);
  if (C_out) memcpy(C_out, C, sizeof(double) * (size_t)k * k);
  free(Y); free(Q); free(R); free(C); free(w); free(P);
  return rc < 0 ? -1 : r;
}

/* ------------------------------------------------------------------------ */
/* Thin SVD by one-sided (Hestenes) Jacobi: the "full SVD of B^T" step of    */
/* Alg. 2.                                                                   */
/* ------------------------------------------------------------------------ */

/* A (m x n, m >= n) = U diag(s) V^T with s descending, U (m x n) orthonormal
 * columns (a zero singular value leaves a zero column), V (n x n) orthogonal.
 * Column pairs (p, q) of a working copy W of A are rotated, W <- W J, until
 * every pair is orthogonal to tol relative to the product of their norms;
 * J is the plane rotation that zeroes the (p, q) entry of W^T W (the same 2x2
 * symmetric Schur step as the two-sided Jacobi above). At the end s_j = |w_j|,
 * U_j = w_j / s_j and V = the accumulated rotations. Returns the number of
 * sweeps, or -1 if max_sweeps was reached first. */
int orc_svd_jacobi(int m, int n, const double* A, double* U, double* s, double* V, int max_sweeps, double tol) {
  double* W = (double*)malloc(sizeof(double) * (size_t)m * n);
  memcpy(W, A, sizeof(double) * (size_t)m * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
  int sweeps = 0, converged = 0;
  while (sweeps < max_sweeps) {
    int rotated = 0;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int i = 0; i < m; ++i) {
          const double wp = W[(size_t)i * n + p], wq = W[(size_t)i * n + q];
          a += wp * wp;
          b += wq * wq;
          c += wp * wq;
        }
        if (a == 0.0 || b == 0.0 || fabs(c) <= tol * sqrt(a * b)) continue;
        rotated = 1;
        double zeta = (b - a) / (2.0 * c);
        double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
        for (int i = 0; i < m; ++i) { /* W <- W J */
          const double wp = W[(size_t)i * n + p], wq = W[(size_t)i * n + q];
          W[(size_t)i * n + p] = cs * wp - sn * wq;
          W[(size_t)i * n + q] = sn * wp + cs * wq;
        }
        for (int i = 0; i < n; ++i) { /* V <- V J */
          const double vp = V[(size_t)i * n + p], vq = V[(size_t)i * n + q];
          V[(size_t)i * n + p] = cs * vp - sn * vq;
          V[(size_t)i * n + q] = sn * vp + cs * vq;
        }
      }
    }
    ++sweeps;
    if (!rotated) { converged = 1; break; }
  }
  for (int j = 0; j < n; ++j) {
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += W[(size_t)i * n + j] * W[(size_t)i * n + j];
    s[j] = sqrt(nrm);
    for (int i = 0; i < m; ++i) U[(size_t)i * n + j] = s[j] > 0.0 ? W[(size_t)i * n + j] / s[j] : 0.0;
  }
  /* stable descending order of s, applied to the columns of U and V */
  int* idx = (int*)malloc(sizeof(int) * (size_t)n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 1; i < n; ++i) {
    int v = idx[i], j = i - 1;
    while (j >= 0 && s[idx[j]] < s[v]) { idx[j + 1] = idx[j]; --j; }
    idx[j + 1] = v;
  }
  double* st = (double*)malloc(sizeof(double) * (size_t)n);
  double* Ut = (double*)malloc(sizeof(double) * (size_t)m * n);
  double* Vt = (double*)malloc(sizeof(double) * (size_t)n * n);
  for (int j = 0; j < n; ++j) {
    st[j] = s[idx[j]];
    for (int i = 0; i < m; ++i) Ut[(size_t)i * n + j] = U[(size_t)i * n + idx[j]];
    for (int i = 0; i < n; ++i) Vt[(size_t)i * n + j] = V[(size_t)i * n + idx[j]];
  }
  memcpy(s, st, sizeof(double) * (size_t)n);
  memcpy(U, Ut, sizeof(double) * (size_t)m * n);
  memcpy(V, Vt, sizeof(double) * (size_t)n * n);
  free(idx); free(st); free(Ut); free(Vt); free(W);
  return converged ? sweeps : -1;
}

/* ------------------------------------------------------------------------ */
/* Randomized SVD of a symmetric PSD factor: Alg. 2 (RSVD) with the power    */
/* iterations of Sec. 2.2, as RS-KFAC (Alg. 4) uses it, returning V~.        */
/* ------------------------------------------------------------------------ */

/* X: d x d symmetric PSD factor; Omega: d x k (k = r + p). Steps: Y = X Omega;
 * Q R = QR(Y); q times: Y = X Q, Q R = QR(Y); B = Q^T X (k x d); full SVD of
 * B^T = U' diag(s) W'^T (one-sided Jacobi), so B = W' diag(s) U'^T: the left
 * singular vectors of B are U_B = W' and its right singular vectors are
 * V_B = U'. Outputs V~ = V_B[:, :r] (d x r), S~ = s[:r] and, when Ut is not
 * NULL, U~ = Q U_B[:, :r] (d x r). When k >= d the factor is diagonalised
 * directly (V~ = U~ = its leading eigenvectors, S~ = its eigenvalues). Returns
 * r_eff = min(r, d), or -1 if a Jacobi solve did not converge. */
int orc_rsvd(int d, const double* X, int k, const double* Omega, int q, int r, double* Vr, double* S, double* Ut) {
  if (r > d) r = d;
  if (k >= d) {
    double* w = (double*)malloc(sizeof(double) * (size_t)d);
    double* E = (double*)malloc(sizeof(double) * (size_t)d * d);
    int rc = orc_jacobi_eigh(d, X, w, E, 100, 1e-15);
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < r; ++j) {
        Vr[(size_t)i * r + j] = E[(size_t)i * d + j];
        if (Ut) Ut[(size_t)i * r + j] = E[(size_t)i * d + j];
      }
    for (int j = 0; j < r; ++j) S[j] = w[j];
    free(w); free(E);
    return rc < 0 ? -1 : r;
  }
  double* Y = (double*)malloc(sizeof(double) * (size_t)d * k);
  double* Q = (double*)malloc(sizeof(double) * (size_t)d * k);
  double* R = (double*)malloc(sizeof(double) * (size_t)k * k);
  double* Bt = (double*)malloc(sizeof(double) * (size_t)d * k);
  double* Us = (double*)malloc(sizeof(double) * (size_t)d * k);
  double* s = (double*)malloc(sizeof(double) * (size_t)k);
  double* Ws = (double*)malloc(sizeof(double) * (size_t)k * k);
  orc_matmul(d, k, d, X, 0, Omega, 0, Y);            /* Y = X Omega          */
  orc_qr(d, k, Y, Q, R);                             /* Q R = QR_decomp(Y)   */
  for (int it = 0; it < q; ++it) {                   /* power iterations     */
    orc_matmul(d, k, d, X, 0, Q, 0, Y);
    orc_qr(d, k, Y, Q, R);
  }
  orc_matmul(d, k, d, X, 1, Q, 0, Bt);               /* B^T = X^T Q (d x k)  */
  int rc = orc_svd_jacobi(d, k, Bt, Us, s, Ws, 100, 1e-15);
  for (int i = 0; i < d; ++i)                        /* V~ = V_B[:, :r]      */
    for (int j = 0; j < r; ++j) Vr[(size_t)i * r + j] = Us[(size_t)i * k + j];
  for (int j = 0; j < r; ++j) S[j] = s[j];
  if (Ut) {                                          /* U~ = Q U_B[:, :r]    */
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < r; ++j) {
        double acc = 0.0;
        for (int t = 0; t < k; ++t) acc += Q[(size_t)i * k + t] * Ws[(size_t)t * k + j];
        Ut[(size_t)i * r + j] = acc;
      }
  }
  free(Y); free(Q); free(R); free(Bt); free(Us); free(s); free(Ws);
  return rc < 0 ? -1 : r;
}

/* ------------------------------------------------------------------------ */
/* Damped low-rank inverse, Eq. (13): (U D U^T + lam I)^-1 = U diag(c) U^T + */
/* I / lam with c_i = 1/(D_i + lam) - 1/lam.                                 */
/* ------------------------------------------------------------------------ */

void orc_damped_coef(int r, const double* D, double lam, double* coef) {
  for (int i = 0; i < r; ++i) {
    double di = D[i] > 0.0 ? D[i] : 0.0; /* clamp round-off negatives */
    coef[i] = 1.0 / (di + lam) - 1.0 / lam;
  }
}

/* ------------------------------------------------------------------------ */
/* Preconditioner apply, Alg. 4 (the M and S updates; Alg. 5 feeds it U~ in  */
/* place of V~): M = J U_a diag(c_a) U_a^T + J/lam,                          */
/*               S = U_g diag(c_g) U_g^T M + M/lam.                          */
/* J = Mat(g) is d_g x d_a; U_a is d_a x r_a; U_g is d_g x r_g.              */
/* ------------------------------------------------------------------------ */

void orc_precondition(int dg, int da, const double* J, const double* Ua, const double* ca, int ra,
                      const double* Ug, const double* cg, int rg, double lam, double* S) {
  double* T = (double*)malloc(sizeof(double) * (size_t)dg * (ra > 0 ? ra : 1));
  double* M = (double*)malloc(sizeof(double) * (size_t)dg * da);
  double* T2 = (double*)malloc(sizeof(double) * (size_t)(rg > 0 ? rg : 1) * da);
  orc_matmul(dg, ra, da, J, 0, Ua, 0, T);            /* T = J U_a            */
  for (int i = 0; i < dg; ++i)
    for (int j = 0; j < ra; ++j) T[(size_t)i * ra + j] *= ca[j];
  orc_matmul(dg, da, ra, T, 0, Ua, 1, M);            /* T diag(c_a) U_a^T    */
  for (size_t i = 0; i < (size_t)dg * da; ++i) M[i] += J[i] / lam;
  orc_matmul(rg, da, dg, Ug, 1, M, 0, T2);           /* T2 = U_g^T M         */
  for (int i = 0; i < rg; ++i)
    for (int j = 0; j < da; ++j) T2[(size_t)i * da + j] *= cg[i];
  orc_matmul(dg, da, rg, Ug, 0, T2, 0, S);           /* U_g diag(c_g) T2     */
  for (size_t i = 0; i < (size_t)dg * da; ++i) S[i] += M[i] / lam;
  free(T); free(M); free(T2);
}

/* Selected columns of the same S (for factor sizes where the full product  */
/* is too slow for a test): column c of M = J (U_a diag(c_a) U_a^T + I/lam)  */
/* is J v + J[:, c]/lam with v = U_a (c_a o U_a[c, :]); column c of S is     */
/* U_g (c_g o U_g^T m) + m/lam. Output S_cols is d_g x ncols (column j of    */
/* it = column cols[j] of S).                                                */
void orc_precondition_cols(int dg, int da, const double* J, const double* Ua, const double* ca, int ra,
                           const double* Ug, const double* cg, int rg, double lam, int ncols, const int* cols,
                           double* S_cols) {
#pragma omp parallel for schedule(dynamic, 1) if (ncols > 1)
  for (int jc = 0; jc < ncols; ++jc) {
    double* v = (double*)malloc(sizeof(double) * (size_t)da);
    double* m = (double*)malloc(sizeof(double) * (size_t)dg);
    double* t = (double*)malloc(sizeof(double) * (size_t)(rg > 0 ? rg : 1));
    const int c = cols[jc];
    for (int i = 0; i < da; ++i) {                     /* v = U_a (c_a o U_a[c, :]) */
      double s = 0.0;
      for (int l = 0; l < ra; ++l) s += Ua[(size_t)i * ra + l] * ca[l] * Ua[(size_t)c * ra + l];
      v[i] = s;
    }
    for (int i = 0; i < dg; ++i) {                     /* m = J v + J[:, c] / lam */
      double s = 0.0;
      for (int l = 0; l < da; ++l) s += J[(size_t)i * da + l] * v[l];
      m[i] = s + J[(size_t)i * da + c] / lam;
    }
    for (int l = 0; l < rg; ++l) {                     /* t = c_g o (U_g^T m) */
      double s = 0.0;
      for (int i = 0; i < dg; ++i) s += Ug[(size_t)i * rg + l] * m[i];
      t[l] = cg[l] * s;
    }
    for (int i = 0; i < dg; ++i) {                     /* S[:, c] = U_g t + m / lam */
      double s = 0.0;
      for (int l = 0; l < rg; ++l) s += Ug[(size_t)i * rg + l] * t[l];
      S_cols[(size_t)i * ncols + jc] = s + m[i] / lam;
    }
    free(v); free(m); free(t);
  }
}

/* ------------------------------------------------------------------------ */
/* Exact damped Kronecker inverse apply through full eigendecompositions:    */
/* Alg. 1 (eigendecomposition, then the M and S updates) with the identity   */
/* of Sec. 2.1,                                                               */
/* S = (G + lam I)^-1 J (A + lam I)^-1.                                      */
/* ------------------------------------------------------------------------ */

int orc_exact_apply(int dg, int da, const double* J, const double* Fa, const double* Fg, double lam, double* S) {
  double* wa = (double*)malloc(sizeof(double) * (size_t)da);
  double* Va = (double*)malloc(sizeof(double) * (size_t)da * da);
  double* wg = (double*)malloc(sizeof(double) * (size_t)dg);
  double* Vg = (double*)malloc(sizeof(double) * (size_t)dg * dg);
  double* T = (double*)malloc(sizeof(double) * (size_t)dg * da);
  double* M = (double*)malloc(sizeof(double) * (size_t)dg * da);
  int rc1 = orc_jacobi_eigh(da, Fa, wa, Va, 100, 1e-15);
  int rc2 = orc_jacobi_eigh(dg, Fg, wg, Vg, 100, 1e-15);
  orc_matmul(dg, da, da, J, 0, Va, 0, T);            /* J U_A                */
  for (int i = 0; i < dg; ++i)
    for (int j = 0; j < da; ++j) T[(size_t)i * da + j] /= (wa[j] + lam);
  orc_matmul(dg, da, da, T, 0, Va, 1, M);            /* M = J U_A (D+lam)^-1 U_A^T */
  orc_matmul(dg, da, dg, Vg, 1, M, 0, T);            /* U_G^T M              */
  for (int i = 0; i < dg; ++i)
    for (int j = 0; j < da; ++j) T[(size_t)i * da + j] /= (wg[i] + lam);
  orc_matmul(dg, da, dg, Vg, 0, T, 0, S);            /* S = U_G (D+lam)^-1 U_G^T M */
  free(wa); free(Va); free(wg); free(Vg); free(T); free(M);
  return (rc1 < 0 || rc2 < 0) ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Proposition 3.1, Eq. (7): at most min(r_eps n_M, d_M) eigenvalues of the  */
/* EA factor exceed eps * lambda_max, r_eps = ceil(log(alpha eps)/log(rho)). */
/* ------------------------------------------------------------------------ */

long orc_rank_bound(double eps, double alpha, double rho, long n_m, long d_m) {
  long r_eps = (long)ceil(log(alpha * eps) / log(rho));
  long b = r_eps * n_m;
  return b < d_m ? b : d_m;
}
