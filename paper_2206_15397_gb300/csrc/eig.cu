// Eigensolver for the small projected matrix C = Q^T F Q ("Eigen_decomp" of
// Alg. 3), and for whole factors with d <= k.
//
//  1. eig_onesided_f32: one CTA per matrix. C + s I (s a small PD shift) is
//     Cholesky-factored in FP32 in shared memory, C + s I = L L^T, and the
//     columns of W = L are made mutually orthogonal by one-sided (Hestenes)
//     Jacobi rotations W <- W J in a round-robin parallel ordering (one warp per
//     column pair). Since W W^T = C + s I is invariant, at convergence the unit
//     columns of W are eigenvectors of C and |w_j|^2 - s its eigenvalues. Only
//     one k x k FP32 matrix is stored (k <= 238 fits in shared memory).
//  2. eig_refine_f64: one FP64 refinement step of all eigenpairs (Ogita and
//     Aishima, "Iterative refinement for symmetric eigenvalue decomposition",
//     2018): from R = I - X^T X and S = X^T C X, lam_i = S_ii / (1 - R_ii) and
//     X <- X + X E with E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i) for
//     separated pairs, R_ij / 2 otherwise. The products are FP64 GEMMs spread
//     over many CTAs; it lifts FP32-accurate pairs to near FP64 accuracy.
//  3. eig_select: descending stable sort, leading r pairs, damping coefficients.
#include "common.cuh"

namespace kfac {
namespace {

constexpr int EIG_THREADS = 512;
constexpr int EIG_WARPS = EIG_THREADS / 32;
constexpr int EIG_SMEM_MAX = kSmemOptin;

__device__ __forceinline__ float warp_sum_bcast(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);  // one value for every lane
}

__global__ void __launch_bounds__(EIG_THREADS) k_eig_onesided(const double* __restrict__ C, int k, double shift_rel,
                                                               int max_sweeps, float tol, double* __restrict__ X,
                                                               double* __restrict__ lam, float* gscratch, int use_smem,
                                                               int* flags, unsigned long long* stats) {
  extern __shared__ __align__(16) float esm[];
  float* W = use_smem ? esm : gscratch;  // column-major: W[j * k + i]
  __shared__ double s_trace, s_shift;
  __shared__ int s_bad, s_count;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid < 32) {
    double t = 0.0;
    for (int i = tid; i < k; i += 32) t += C[(size_t)i * k + i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (tid == 0) {
      s_trace = t;
      s_shift = fmax(shift_rel * fabs(t), 1e-30);
    }
  }
  __syncthreads();
  if (!isfinite(s_trace)) {
    if (tid == 0) raise_flag(flags, KFAC_FLAG_NONFINITE);
    for (long long e = tid; e < (long long)k * k; e += EIG_THREADS) X[e] = ((e / k) == (e % k)) ? 1.0 : 0.0;
    for (int i = tid; i < k; i += EIG_THREADS) lam[i] = 0.0;
    return;
  }

  // ---- FP32 Cholesky of C + s I, growing s on breakdown --------------------
  for (int attempt = 0;; ++attempt) {
    const double sh = s_shift;
    for (long long e = tid; e < (long long)k * k; e += EIG_THREADS) {
      int j = (int)(e / k), i = (int)(e % k);
      W[e] = (i >= j) ? (float)(C[(size_t)i * k + j] + (i == j ? sh : 0.0)) : 0.0f;
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int j = 0; j < k; ++j) {
      if (tid == 0) {
        float p = W[(size_t)j * k + j];
        if (!(p > 0.0f) || !isfinite(p)) s_bad = 1;
        else W[(size_t)j * k + j] = sqrtf(p);
      }
      __syncthreads();
      if (s_bad) break;
      const float ljj = W[(size_t)j * k + j];
      for (int i = j + 1 + tid; i < k; i += EIG_THREADS) W[(size_t)j * k + i] /= ljj;
      __syncthreads();
      const int n = k - j - 1;  // trailing (i, l) with j < l <= i < k
      for (long long e = tid; e < (long long)n * n; e += EIG_THREADS) {
        int l = j + 1 + (int)(e / n), i = j + 1 + (int)(e % n);
        if (i >= l) W[(size_t)l * k + i] -= W[(size_t)j * k + i] * W[(size_t)j * k + l];
      }
      __syncthreads();
    }
    if (!s_bad) break;
    if (attempt >= 4) {
      if (tid == 0) raise_flag(flags, KFAC_FLAG_CHOL_FAILED);
      break;
    }
    if (tid == 0) {
      s_shift = fmax(s_shift * 100.0, 1e-6 * fabs(s_trace));
      raise_flag(flags, KFAC_FLAG_EIG_SHIFTED);
    }
    __syncthreads();
  }

  // ---- one-sided Jacobi, round-robin ordering -------------------------------
  // Players 0..m-1 (m even, a phantom column when k is odd). Round r pairs
  // (r, m-1) and ((r+p) mod (m-1), (r-p) mod (m-1)) for p = 1..m/2-1; m-1
  // rounds visit every pair once.
  const int m = k + (k & 1);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_count = 0;
    __syncthreads();
    for (int r = 0; r < m - 1; ++r) {
      for (int p = warp; p < m / 2; p += EIG_WARPS) {
        int a, b;
        if (p == 0) { a = r; b = m - 1; }
        else { a = (r + p) % (m - 1); b = (r - p + (m - 1)) % (m - 1); }
        if (a >= k || b >= k) continue;
        float* wa = W + (size_t)a * k;
        float* wb = W + (size_t)b * k;
        float al = 0.f, be = 0.f, ga = 0.f;
        for (int i = lane; i < k; i += 32) {
          float x = wa[i], y = wb[i];
          al = fmaf(x, x, al);
          be = fmaf(y, y, be);
          ga = fmaf(x, y, ga);
        }
        al = warp_sum_bcast(al);
        be = warp_sum_bcast(be);
        ga = warp_sum_bcast(ga);
        if (ga != 0.0f && fabsf(ga) > tol * sqrtf(al * be)) {
          float zeta = (be - al) / (2.0f * ga);
          float t = (zeta >= 0.0f ? 1.0f : -1.0f) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
          float cs = rsqrtf(1.0f + t * t), sn = cs * t;
          for (int i = lane; i < k; i += 32) {
            float x = wa[i], y = wb[i];
            wa[i] = cs * x - sn * y;
            wb[i] = sn * x + cs * y;
          }
          if (lane == 0) atomicAdd(&s_count, 1);
        }
      }
      __syncthreads();
    }
    if (s_count == 0) break;
  }
  if (sweep >= max_sweeps && tid == 0) raise_flag(flags, KFAC_FLAG_EIG_NOCONV);
  if (stats && tid == 0) {
    atomicAdd(stats + STAT_SWEEPS, (unsigned long long)(sweep < max_sweeps ? sweep + 1 : sweep));
    atomicAdd(stats + STAT_EIG_SOLVES, 1ull);
  }

  // ---- eigenpairs: lam_j = |w_j|^2 - s, x_j = w_j / |w_j| -------------------
  const double sh = s_shift;
  for (int j = warp; j < k; j += EIG_WARPS) {
    const float* wj = W + (size_t)j * k;
    double n2 = 0.0;
    for (int i = lane; i < k; i += 32) n2 += (double)wj[i] * (double)wj[i];
    for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    n2 = __shfl_sync(0xffffffffu, n2, 0);
    double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
    for (int i = lane; i < k; i += 32) X[(size_t)i * k + j] = (double)wj[i] * inv;
    if (lane == 0) lam[j] = n2 - sh;
  }
}

// Refinement combine (one CTA): E from R = I - X^T X (given as XtX) and S.
__global__ void __launch_bounds__(1024) k_refine_combine(const double* __restrict__ C, const double* __restrict__ XtX,
                                                          const double* __restrict__ S, int k, double* __restrict__ E,
                                                          double* __restrict__ lam, int* flags) {
  __shared__ double red[3][32];
  __shared__ double s_delta;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < k; i += blockDim.x) {
    double xx = XtX[(size_t)i * k + i];
    lam[i] = S[(size_t)i * k + i] / xx;  // S_ii / (1 - R_ii)
  }
  __syncthreads();
  double a = 0.0, b = 0.0, c = 0.0;  // ||S - diag(lam)||_F^2, ||C||_F^2, ||R||_F^2
  for (long long e = tid; e < (long long)k * k; e += blockDim.x) {
    int i = (int)(e / k), j = (int)(e % k);
    double sv = S[e] - (i == j ? lam[i] : 0.0);
    double rv = (i == j ? 1.0 : 0.0) - XtX[e];
    a += sv * sv;
    b += C[e] * C[e];
    c += rv * rv;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if (lane == 0) { red[0][warp] = a; red[1][warp] = b; red[2][warp] = c; }
  __syncthreads();
  if (tid == 0) {
    double A = 0, Bn = 0, Cn = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) { A += red[0][w]; Bn += red[1][w]; Cn += red[2][w]; }
    s_delta = 2.0 * (sqrt(A) + sqrt(Bn) * sqrt(Cn));
    if (!isfinite(s_delta)) raise_flag(flags, KFAC_FLAG_NONFINITE);
  }
  __syncthreads();
  const double delta = s_delta;
  for (long long e = tid; e < (long long)k * k; e += blockDim.x) {
    int i = (int)(e / k), j = (int)(e % k);
    double rij = (i == j ? 1.0 : 0.0) - XtX[e];
    double v;
    if (i == j) {
      v = 0.5 * rij;
    } else {
      double gap = lam[j] - lam[i];
      v = (fabs(gap) > delta) ? (S[e] + lam[j] * rij) / gap : 0.5 * rij;
    }
    E[e] = v;
  }
}

__global__ void __launch_bounds__(1024) k_eig_select(const double* __restrict__ X, const double* __restrict__ lam,
                                                      int k, int r, float lambda, float* __restrict__ P32,
                                                      float* __restrict__ D, float* __restrict__ coef,
                                                      float* __restrict__ Uout, long long ldu) {
  extern __shared__ int order[];  // order[rank] = index
  const int tid = threadIdx.x;
  for (int i = tid; i < k; i += blockDim.x) {
    double li = lam[i];
    if (li != li) li = -INFINITY;
    int rk = 0;
    for (int j = 0; j < k; ++j) {
      double lj = lam[j];
      if (lj != lj) lj = -INFINITY;
      rk += (lj > li) || (lj == li && j < i);
    }
    order[rk] = i;
  }
  __syncthreads();
  for (int t = tid; t < r; t += blockDim.x) {
    double v = lam[order[t]];
    double dv = v > 0.0 ? v : 0.0;
    if (D) D[t] = (float)v;
    if (coef) coef[t] = (float)(1.0 / (dv + (double)lambda) - 1.0 / (double)lambda);
  }
  for (long long e = tid; e < (long long)k * r; e += blockDim.x) {
    int row = (int)(e / r), t = (int)(e % r);
    float v = (float)X[(size_t)row * k + order[t]];
    if (P32) P32[e] = v;
    if (Uout) Uout[(long long)row * ldu + t] = v;
  }
}

}  // namespace

cudaError_t eig_onesided_f32(const double* C, int k, double shift_rel, int max_sweeps, float tol, double* X,
                             double* lam, float* gscratch, int* flags, unsigned long long* stats, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_eig_onesided, cudaFuncAttributeMaxDynamicSharedMemorySize, EIG_SMEM_MAX);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  size_t need = sizeof(float) * (size_t)k * k;
  int use_smem = need <= (size_t)EIG_SMEM_MAX - 1024;
  k_eig_onesided<<<1, EIG_THREADS, use_smem ? need : 0, s>>>(C, k, shift_rel, max_sweeps, tol, X, lam, gscratch,
                                                             use_smem, flags, stats);
  note_launch();
  return cudaGetLastError();
}

cudaError_t eig_refine_f64(const double* C, int k, double* X, double* lam, double* work, int* flags, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  const size_t kk = (size_t)k * k;
  double* XtX = work;
  double* CX = work + kk;
  double* S = work + 2 * kk;
  double* E = work + 3 * kk;
  double* Xn = work + 4 * kk;
  GemmDesc<double> g = {};
  g.M = k; g.N = k; g.K = k; g.alpha = 1.0; g.beta = 0.0; g.zsplit = 1;
  // XtX = X^T X
  g.A = X; g.sam = 1; g.sak = k; g.B = X; g.sbn = 1; g.sbk = k; g.D = XtX; g.ldd = k;
  cudaError_t e = gemm_simt_f64(g, s);
  if (e != cudaSuccess) return e;
  // CX = C X
  g.A = C; g.sam = k; g.sak = 1; g.B = X; g.sbn = 1; g.sbk = k; g.D = CX; g.ldd = k;
  if ((e = gemm_simt_f64(g, s)) != cudaSuccess) return e;
  // S = X^T (C X)
  g.A = X; g.sam = 1; g.sak = k; g.B = CX; g.sbn = 1; g.sbk = k; g.D = S; g.ldd = k;
  if ((e = gemm_simt_f64(g, s)) != cudaSuccess) return e;
  k_refine_combine<<<1, 1024, 0, s>>>(C, XtX, S, k, E, lam, flags);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // Xn = X + X E
  g.A = X; g.sam = k; g.sak = 1; g.B = E; g.sbn = 1; g.sbk = k; g.D = Xn; g.ldd = k; g.beta = 1.0; g.C0 = X;
  g.ldc = k;
  if ((e = gemm_simt_f64(g, s)) != cudaSuccess) return e;
  return cudaMemcpyAsync(X, Xn, kk * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

cudaError_t eig_select(const double* X, const double* lam, int k, int r, float lambda, float* P32, float* D,
                       float* coef, float* Uout, long long ldu, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_eig_select<<<1, 1024, sizeof(int) * k, s>>>(X, lam, k, r, lambda, P32, D, coef, Uout, ldu);
  note_launch();
  return cudaGetLastError();
}

}  // namespace kfac
