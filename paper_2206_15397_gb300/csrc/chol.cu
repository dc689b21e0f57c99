// FP64 Cholesky of the CholeskyQR Gram matrix on one thread-block cluster.
//
// FP64 runs at about 2 FMA/clock/SM on this part, so a k x k Cholesky (k^3/3
// FMA) is spread over up to 16 CTAs of a cluster. Rows are distributed
// cyclically (row i lives in CTA i % NC, in its shared memory). A blocked
// right-looking factorisation with panel width B runs in lock-step:
//   (a) the owners of the diagonal-block rows broadcast them into every CTA
//       (distributed shared memory stores);            cluster barrier
//   (b) every CTA factors the B x B diagonal block redundantly (identical data,
//       identical code -> identical pivots and breakdown decisions), solves its
//       own panel rows L21 = A21 L11^-T and broadcasts them;   cluster barrier
//   (c) every CTA applies the rank-B update to its own trailing rows.
// Panel buffers are double-buffered so (c) of one panel never races with (b)
// of the next. There are no spin waits: only hardware cluster barriers, taken
// the same number of times by every CTA.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace kfac {
namespace {

constexpr int CHOL_THREADS = 256;
constexpr int CHOL_ATTEMPTS = 4;

// 1/sqrt(x) for x > 0 in FP64: an FP32 estimate refined by two Newton steps
// y <- y (3 - x y^2) / 2 (each roughly doubles the number of correct bits:
// ~2^-23 -> 2^-46 -> rounding). Far cheaper here than FP64 sqrt + divide.
__device__ __forceinline__ double rsqrt_newton(double x) {
  double y = (double)rsqrtf((float)x);
  y = y * fma(-0.5 * x * y, y, 1.5);
  y = y * fma(-0.5 * x * y, y, 1.5);
  return y;
}

struct CholSmem {
  double* W;      // nloc x k, own rows (row-major, lower part used)
  double* D;      // B x B diagonal block (replicated in every CTA)
  double* dinv;   // B reciprocals of diag(L11)
  double* P[2];   // panel L21, column-major B x k: P[t * k + i] (replicated, double-buffered)
  int* flag;      // breakdown flag
};

__global__ void __launch_bounds__(CHOL_THREADS, 1) k_chol_cluster(const double* __restrict__ G, int k, int B,
                                                                   int nloc, double shift_rel,
                                                                   float* __restrict__ L32, int* flags,
                                                                   unsigned long long* stats) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int NC = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;

  CholSmem sm;
  double* base = reinterpret_cast<double*>(smem_raw);
  sm.W = base;
  sm.D = sm.W + (size_t)nloc * k;
  sm.dinv = sm.D + B * B;
  sm.P[0] = sm.dinv + B;
  sm.P[1] = sm.P[0] + (size_t)k * B;
  sm.flag = reinterpret_cast<int*>(sm.P[1] + (size_t)k * B);

  // Trace (identical in every CTA: same reads, same order).
  __shared__ double s_trace;
  if (tid < 32) {  // fixed summation order: lane-strided partial sums, then a fixed shuffle tree
    double t = 0.0;
    for (int i = tid; i < k; i += 32) t += G[(size_t)i * k + i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (tid == 0) s_trace = t;
  }
  __syncthreads();
  const double trace = s_trace;
  const bool finite_in = isfinite(trace) && trace > 0.0;
  const double piv_min = 1e-13 * trace;

  // shift_rel > 0: relative to trace(G); shift_rel < 0: |shift_rel| times the
  // mean diagonal trace(G) / k.
  double shift = shift_rel > 0.0 ? shift_rel * trace : (shift_rel < 0.0 ? -shift_rel * trace / k : 0.0);
  int ok = 0;
  for (int attempt = 0; attempt < CHOL_ATTEMPTS && finite_in; ++attempt) {
    if (attempt > 0) {
      shift = fmax(shift, 1e-7 * trace) * 100.0;
      if (rank == 0 && tid == 0) {
        raise_flag(flags, KFAC_FLAG_CHOL_SHIFTED);
        if (stats) atomicAdd(stats + STAT_CHOL_RETRY, 1ull);
      }
    }
    // Load own rows (lower triangle, shifted diagonal).
    for (int li = 0; li < nloc; ++li) {
      int i = li * NC + rank;
      for (int j = tid; j < k; j += CHOL_THREADS) {
        double v = 0.0;
        if (i < k && j <= i) v = G[(size_t)i * k + j] + (i == j ? shift : 0.0);
        sm.W[(size_t)li * k + j] = v;
      }
    }
    if (tid == 0) *sm.flag = 0;
    __syncthreads();
    cluster.sync();  // also: every CTA has started before the first remote store

    int buf = 0;
    int bad = 0;
    for (int j0 = 0; j0 < k; j0 += B) {
      const int jb = min(B, k - j0);
      // (a) owners broadcast the rows of the diagonal block (lower part).
      for (int e = tid; e < jb * jb; e += CHOL_THREADS) {
        const int u = e / jb, t = e % jb, i = j0 + u;
        if (i % NC != rank) continue;
        const double v = (t <= u) ? sm.W[(size_t)(i / NC) * k + j0 + t] : 0.0;
        for (int q = 0; q < NC; ++q) cluster.map_shared_rank(sm.D, q)[u * B + t] = v;
      }
      cluster.sync();
      // (b) factor the diagonal block in place, all threads (same data and code
      //     in every CTA -> identical pivots and breakdown decisions).
      for (int t = 0; t < jb; ++t) {
        const double piv = sm.D[t * B + t];
        if (!(isfinite(piv) && piv > piv_min)) { bad = 1; break; }
        // FP64 issues per warp instruction whatever the active lanes, so the
        // reciprocal square root is evaluated by one thread only.
        __syncthreads();  // everyone has read D[t][t]
        if (tid == 0) {
          const double y = rsqrt_newton(piv);
          sm.D[t * B + t] = piv * y;
          sm.dinv[t] = y;
        }
        __syncthreads();
        const double y = sm.dinv[t];
        for (int u = t + 1 + tid; u < jb; u += CHOL_THREADS) sm.D[u * B + t] *= y;
        __syncthreads();
        const int n = jb - t - 1;  // trailing (u, v), t < v <= u < jb
        for (int e = tid; e < n * n; e += CHOL_THREADS) {
          const int u = t + 1 + e / n, v = t + 1 + e % n;
          if (v <= u) sm.D[u * B + v] = fma(-sm.D[u * B + t], sm.D[v * B + t], sm.D[u * B + v]);
        }
        __syncthreads();
      }
      if (bad) break;  // identical decision in every CTA; no remote stores pending
      // (b') own diagonal rows take L11; own rows below solve L21 = A21 L11^-T
      //      by forward substitution (thread per row) and broadcast the panel.
      for (int e = tid; e < jb * jb; e += CHOL_THREADS) {
        const int u = e / jb, t = e % jb, i = j0 + u;
        if (i % NC == rank && t <= u) sm.W[(size_t)(i / NC) * k + j0 + t] = sm.D[u * B + t];
      }
      const int first = j0 + jb;
      int li0 = (first - rank + NC - 1) / NC;
      if (li0 < 0) li0 = 0;
      const int nrows = nloc - li0;
      double* P = sm.P[buf];
      for (int lr = li0 + tid; lr < nloc; lr += CHOL_THREADS) {
        const int i = lr * NC + rank;
        if (i >= k) continue;
        double* wrow = sm.W + (size_t)lr * k + j0;
        for (int t = 0; t < jb; ++t) {
          double x = wrow[t];
          for (int u = 0; u < t; ++u) x = fma(-wrow[u], sm.D[t * B + u], x);
          x *= sm.dinv[t];
          wrow[t] = x;
          P[(size_t)t * k + i] = x;
        }
      }
      __syncthreads();
      if (NC > 1 && nrows > 0) {
        for (int e = tid; e < nrows * jb; e += CHOL_THREADS) {
          const int lr = li0 + e / jb, t = e % jb, i = lr * NC + rank;
          if (i >= k) continue;
          const double x = P[(size_t)t * k + i];
          for (int q = 0; q < NC; ++q)
            if (q != rank) cluster.map_shared_rank(P, q)[(size_t)t * k + i] = x;
        }
      }
      cluster.sync();
      // (c) trailing update of own rows: W[i][j] -= sum_t L21[i][t] L21[j][t],
      //     first <= j <= i; warp per row, lanes over j (P reads conflict-free).
      for (int lr = li0 + (tid >> 5); lr < nloc; lr += CHOL_THREADS / 32) {
        const int i = lr * NC + rank;
        if (i >= k) continue;
        double* wrow = sm.W + (size_t)lr * k;
        for (int j = first + (tid & 31); j <= i; j += 32) {
          double acc = 0.0;
          for (int t = 0; t < jb; ++t) acc = fma(P[(size_t)t * k + i], P[(size_t)t * k + j], acc);
          wrow[j] -= acc;
        }
      }
      __syncthreads();
      buf ^= 1;
    }
    cluster.sync();
    if (!bad) { ok = 1; break; }
  }

  if (!ok) {
    if (rank == 0 && tid == 0) raise_flag(flags, finite_in ? KFAC_FLAG_CHOL_FAILED : KFAC_FLAG_NONFINITE);
    // Keep downstream finite: L = diag(sqrt(max(G_ii, tiny))).
    for (int li = 0; li < nloc; ++li) {
      int i = li * NC + rank;
      if (i >= k) continue;
      for (int j = tid; j < k; j += CHOL_THREADS) {
        double g = G[(size_t)i * k + i];
        L32[(size_t)i * k + j] = (i == j) ? (float)sqrt(isfinite(g) && g > 1e-30 ? g : 1.0) : 0.0f;
      }
    }
  } else {
    for (int li = 0; li < nloc; ++li) {
      int i = li * NC + rank;
      if (i >= k) continue;
      for (int j = tid; j < k; j += CHOL_THREADS)
        L32[(size_t)i * k + j] = (j <= i) ? (float)sm.W[(size_t)li * k + j] : 0.0f;
    }
  }
  if (stats && rank == 0 && tid == 0) atomicAdd(stats + STAT_CHOL, 1ull);
  cluster.sync();  // no CTA leaves while others may still address its shared memory
}

size_t chol_smem_bytes(int k, int nloc, int B) {
  return sizeof(double) * ((size_t)nloc * k + (size_t)B * B + B + 2 * (size_t)k * B) + 16;
}

}  // namespace

cudaError_t chol_f64_cluster(const double* G, int k, double shift_rel, float* L32, int* flags,
                             unsigned long long* stats, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_chol_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_chol_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemOptin);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  int nc = (k + 15) / 16;
  if (nc > 16) nc = 16;
  if (nc < 1) nc = 1;
  int B = 16;
  int nloc = (k + nc - 1) / nc;
  size_t smem = chol_smem_bytes(k, nloc, B);
  while (smem > (size_t)kSmemOptin && B > 4) {
    B /= 2;
    smem = chol_smem_bytes(k, nloc, B);
  }
  if (smem > (size_t)kSmemOptin) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc, 1, 1);
  cfg.blockDim = dim3(CHOL_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  return cudaLaunchKernelEx(&cfg, k_chol_cluster, G, k, B, nloc, shift_rel, L32, flags, stats);
}


// ---------------------------------------------------------------------------
// Qt = L^-1 Yt: forward substitution with the FP32 lower factor, applied to all
// d columns of Yt at once. Each CTA owns 32 columns and keeps its k x 32 slab of
// the solution in shared memory; rows are processed in blocks of 32: the block
// first receives the contributions of all solved rows (a small GEMM through
// 32 x 32 tiles of L), then its 32 x 32 diagonal block is solved by one warp
// (one lane per column).
namespace {
constexpr int TR_COLS = 32, TR_RB = 32, TR_THREADS = 256;

__global__ void __launch_bounds__(TR_THREADS) k_trsm_lower(const float* __restrict__ L, int k,
                                                            const float* __restrict__ Yt, long long ldy,
                                                            float* __restrict__ Qt, long long ldq, int d) {
  extern __shared__ __align__(16) float tsm[];
  float* X = tsm;                                   // k x TR_COLS
  float* Lt = X + (size_t)k * TR_COLS;              // TR_RB x (TR_RB + 1)
  const int tid = threadIdx.x, c = tid & 31, r0 = tid >> 5;  // 8 row groups
  const int col0 = blockIdx.x * TR_COLS;
  const int col = col0 + c;
  for (int i0 = 0; i0 < k; i0 += TR_RB) {
    const int ib = min(TR_RB, k - i0);
    float acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int ri = r0 + 8 * u;
      acc[u] = (ri < ib && col < d) ? Yt[(long long)(i0 + ri) * ldy + col] : 0.0f;
    }
    for (int m0 = 0; m0 < i0; m0 += TR_RB) {
      for (int e = tid; e < TR_RB * TR_RB; e += TR_THREADS) {
        int a = e / TR_RB, b = e % TR_RB;
        Lt[a * (TR_RB + 1) + b] = (a < ib) ? L[(size_t)(i0 + a) * k + m0 + b] : 0.0f;
      }
      __syncthreads();
#pragma unroll 8
      for (int mm = 0; mm < TR_RB; ++mm) {
        float x = X[(size_t)(m0 + mm) * TR_COLS + c];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fmaf(-Lt[(r0 + 8 * u) * (TR_RB + 1) + mm], x, acc[u]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int ri = r0 + 8 * u;
      if (ri < ib) X[(size_t)(i0 + ri) * TR_COLS + c] = acc[u];
    }
    for (int e = tid; e < TR_RB * TR_RB; e += TR_THREADS) {
      int a = e / TR_RB, b = e % TR_RB;
      Lt[a * (TR_RB + 1) + b] = (a < ib && b < ib) ? L[(size_t)(i0 + a) * k + i0 + b] : 0.0f;
    }
    __syncthreads();
    if (tid < 32) {  // lane c solves its column through the diagonal block
      for (int t = 0; t < ib; ++t) {
        float x = X[(size_t)(i0 + t) * TR_COLS + c];
        for (int u = 0; u < t; ++u) x = fmaf(-Lt[t * (TR_RB + 1) + u], X[(size_t)(i0 + u) * TR_COLS + c], x);
        X[(size_t)(i0 + t) * TR_COLS + c] = x / Lt[t * (TR_RB + 1) + t];
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int ri = r0 + 8 * u;
      if (ri < ib && col < d) Qt[(long long)(i0 + ri) * ldq + col] = X[(size_t)(i0 + ri) * TR_COLS + c];
    }
  }
}
}  // namespace

cudaError_t trsm_lower_f32(const float* L, int k, const float* Yt, long long ldy, float* Qt, long long ldq, int d,
                           cudaStream_t s) {
  if (k <= 0 || d <= 0) return cudaSuccess;
  size_t smem = sizeof(float) * ((size_t)k * TR_COLS + TR_RB * (TR_RB + 1));
  if (smem > (size_t)kSmemOptin) return cudaErrorInvalidValue;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_trsm_lower, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemOptin);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  k_trsm_lower<<<(d + TR_COLS - 1) / TR_COLS, TR_THREADS, smem, s>>>(L, k, Yt, ldy, Qt, ldq, d);
  note_launch();
  return cudaGetLastError();
}

}  // namespace kfac
