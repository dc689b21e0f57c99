// Cholesky factorisations of the CholeskyQR Grams and of the eigensolver's
// shifted projected matrix, and the triangular solve Q^T = L^-1 Y^T:
//   - k_chol_cta_f32: FP32 on one CTA with the matrix in shared memory, the
//     default for k <= CTA_KMAX (described at the kernel);
//   - k_chol_cluster<T>: FP32 above that size, or FP64 when the options ask
//     for it, on one thread-block cluster (below);
//   - k_trsm_pack / k_trsm_lower_smem / k_trsm_lower: the block solve.
//
// Cluster kernel. FP64 runs at about 2 FMA/clock/SM on this part, so a k x k
// Cholesky (k^3/3 FMA) is spread over up to 16 CTAs of a cluster. Rows are distributed
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
#include "gemm.cuh"

namespace cg = cooperative_groups;

namespace kfac {
namespace {

constexpr int CHOL_THREADS = 256;
constexpr int CHOL_ATTEMPTS = 4;

// 1/sqrt(x) for x > 0 in FP64: an FP32 estimate refined by one Newton step
// y <- y (3 - x y^2) / 2, which squares the relative error (~2^-23 -> ~2^-46):
// far below the accuracy of the FP32-accumulated Gram it factors, and three
// FP64 instructions instead of an FP64 sqrt and divide (an FP64 warp
// instruction costs ~68 cycles on this part whatever its active lanes).
__device__ __forceinline__ double rsqrt_newton(double x) {
  double y = (double)rsqrtf((float)x);
  return y * fma(-0.5 * x * y, y, 1.5);
}
__device__ __forceinline__ float rsqrt_newton(float x) {
  const float y = rsqrtf(x);
  return y * fmaf(-0.5f * x * y, y, 1.5f);
}

// Replacement for a pivot below the floor: the column's original diagonal.
template <typename T>
__device__ __forceinline__ T raised_pivot(const double* G, int k, int j, double shift, T pfloor) {
  const T g = (T)(G[(size_t)j * k + j] + shift);
  return g > pfloor ? g : pfloor;
}

template <typename T>
struct CholSmem {
  T* W;      // nloc x k, own rows (row-major, lower part used)
  T* D;      // B x B diagonal block (replicated in every CTA)
  T* dinv;   // B reciprocals of diag(L11)
  T* Xi;     // B x B inverse of L11 (replicated)
  T* P[2];   // panel L21, column-major B x k: P[t * k + i] (replicated, double-buffered)
  int* flag;     // breakdown flag (non-finite pivot)
  int* clamped;  // a pivot was raised to the floor
};

template <typename T>
__global__ void __launch_bounds__(CHOL_THREADS, 1) k_chol_cluster(const double* __restrict__ G, int k, int B,
                                                                   int nloc, double shift_rel,
                                                                   float* __restrict__ L32, int* flags,
                                                                   unsigned long long* stats, double* shift_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int NC = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;

  CholSmem<T> sm;
  T* base = reinterpret_cast<T*>(smem_raw);
  sm.P[0] = base;  // first: 16-byte aligned (it also stages the FP64 diagonal)
  sm.P[1] = sm.P[0] + (size_t)k * B;
  sm.W = sm.P[1] + (size_t)k * B;
  sm.D = sm.W + (size_t)nloc * k;
  sm.dinv = sm.D + B * B;
  sm.Xi = sm.dinv + B;
  sm.flag = reinterpret_cast<int*>(sm.Xi + B * B);
  sm.clamped = sm.flag + 1;

  // Trace (identical in every CTA: same reads, same order). The diagonal is
  // staged in the (still unused) panel buffer with all loads in flight at once.
  __shared__ double s_trace;
  {
    double* dg = reinterpret_cast<double*>(sm.P[0]);  // k doubles fit in k * B (B >= 4) elements of T
    for (int i = tid; i < k; i += CHOL_THREADS) cp_async8(dg + i, G + (size_t)i * k + i);
    cp_async_wait_all();
    __syncthreads();
    if (tid < 32) {  // fixed summation order: lane-strided partial sums, then a fixed shuffle tree
      double t = 0.0;
      for (int i = tid; i < k; i += 32) t += fabs(dg[i]);
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (tid == 0) s_trace = t;
    }
    __syncthreads();
  }
  const double trace = s_trace;
  // trace: sum of |G_ii| (the trace of a PSD matrix; a scale for the shifts and
  // the floor of any symmetric one). A zero diagonal means the zero matrix
  // (the Gram of a zero sketch, or a zero projected matrix): it is factored
  // exactly as G + 1 I = I I^T (L = I, shift 1).
  const bool finite_in = isfinite(trace) && trace > 0.0;
  const bool zero_in = trace == 0.0;
  // Pivot floor. A pivot below it (the column is, to the Gram's FP32
  // accuracy, in the span of the previous ones) is replaced by the column's
  // original diagonal G_jj + shift (at least the floor): the factor is then
  // the exact Cholesky factor of G + shift I + diag(delta), delta >= 0, which
  // keeps R invertible and span(Y R^-1) = span(Y), and the column's
  // multipliers stay bounded by the rest of the matrix instead of growing by
  // 1/sqrt(floor). The floor is relative to the mean diagonal, above the
  // rounding noise of the FP32-accurate Gram (and of an FP32 factorisation).
  // Should the raised pivots still let the factorisation overflow, the
  // non-finite pivot restarts it with a larger shift.
  const T pfloor = (T)(sizeof(T) == 4 ? fmax(1e-9 * trace, 1e-6 * trace / k) : fmax(1e-13 * trace, 1e-7 * trace / k));

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
    // Load own rows (lower triangle, shifted diagonal), eight independent
    // loads per thread in flight before their stores.
    {
      const int total = nloc * k;
      for (int base = 0; base < total; base += 8 * CHOL_THREADS) {
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int e = base + q * CHOL_THREADS + tid;
          const int li = e / k, j = e - li * k, i = li * NC + rank;
          v[q] = (e < total && i < k && j <= i) ? G[(size_t)i * k + j] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int e = base + q * CHOL_THREADS + tid;
          if (e < total) {
            const int li = e / k, j = e - li * k, i = li * NC + rank;
            sm.W[e] = (T)(v[q] + (i == j ? shift : 0.0));
          }
        }
      }
    }
    if (tid == 0) { *sm.flag = 0; *sm.clamped = 0; }
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
        const T v = (t <= u) ? sm.W[(size_t)(i / NC) * k + j0 + t] : T(0);
        for (int q = 0; q < NC; ++q) cluster.map_shared_rank(sm.D, q)[u * B + t] = v;
      }
      cluster.sync();
      // (b) factor the diagonal block in place and form Xi = L11^-1 beside it
      //     (same data and code in every CTA -> identical pivots and breakdown
      //     decisions). An FP64 warp instruction costs ~68 cycles on its
      //     sub-partition whatever its active lanes, so the element work runs
      //     on warps 0-3 (one per sub-partition) and the chain through the
      //     pivots on one thread of warp 4, one step ahead: while warps 0-3
      //     apply step t's rank-1 update, that thread already holds the next
      //     pivot (updated first) and computes its reciprocal root. Per step t:
      //       A: column t of L and row t of Xi are scaled by y_t = L_tt^-1;
      //          the pivot thread scales L_{t+1,t} and updates A_{t+1,t+1};
      //       B: the trailing triangle {t < v <= u < jb} except (t+1, t+1) and
      //          the Xi rows u > t take the update; the pivot thread checks
      //          A_{t+1,t+1} and writes y_{t+1}.
      //     Triangle entries are enumerated as (u', v') = (jb-1-u, jb-1-v),
      //     u' <= v', ordered by v', so the active set is a prefix on full lanes.
      if (tid < 160) {
        if (tid < 128) {
          for (int e = tid; e < jb * B; e += 128) sm.Xi[e] = T(0);
        } else if (tid == 128) {
          T piv = sm.D[0];
          if (!isfinite(piv)) {
            *sm.flag = 1;
          } else {
            if (!(piv > pfloor)) { piv = raised_pivot(G, k, j0, shift, pfloor); sm.D[0] = piv; *sm.clamped = 1; }
            sm.dinv[0] = rsqrt_newton(piv);
          }
        }
        asm volatile("bar.sync 1, 160;" ::: "memory");
        for (int t = 0; t < jb; ++t) {
          if (*sm.flag) break;  // written before the last barrier: uniform
          const T y = sm.dinv[t];
          if (tid < 128) {
            if (tid == t) sm.D[t * B + t] *= y;  // L_tt = A_tt y_t = sqrt(A_tt)
            else if (tid > t + 1 && tid < jb) sm.D[tid * B + t] *= y;
            if (tid <= t) sm.Xi[t * B + tid] = (tid == t) ? y : sm.Xi[t * B + tid] * y;
          } else if (tid == 128 && t + 1 < jb) {
            const T l = sm.D[(t + 1) * B + t] * y;
            sm.D[(t + 1) * B + t] = l;
            sm.D[(t + 1) * B + t + 1] = fma(-l, l, sm.D[(t + 1) * B + t + 1]);
          }
          asm volatile("bar.sync 1, 160;" ::: "memory");
          const int n = jb - t - 1;
          if (tid < 128) {
            const int ctri = n * (n + 1) / 2, total = ctri + n * (t + 1);
            for (int e = tid; e < total; e += 128) {
              if (e < ctri) {
                const int vp = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f + 1e-4f);
                const int up = e - vp * (vp + 1) / 2;
                const int u = jb - 1 - up, v = jb - 1 - vp;
                if (v == t + 1 && u == t + 1) continue;  // the next pivot: done in A
                sm.D[u * B + v] = fma(-sm.D[u * B + t], sm.D[v * B + t], sm.D[u * B + v]);
              } else {
                const int e2 = e - ctri, u = t + 1 + e2 / (t + 1), c = e2 % (t + 1);
                sm.Xi[u * B + c] = fma(-sm.D[u * B + t], sm.Xi[t * B + c], sm.Xi[u * B + c]);
              }
            }
          } else if (tid == 128 && n > 0) {
            T piv = sm.D[(t + 1) * B + t + 1];
            if (!isfinite(piv)) {
              *sm.flag = 1;
            } else {
              if (!(piv > pfloor)) {
                piv = raised_pivot(G, k, j0 + t + 1, shift, pfloor);
                sm.D[(t + 1) * B + t + 1] = piv;
                *sm.clamped = 1;
              }
              sm.dinv[t + 1] = rsqrt_newton(piv);
            }
          }
          asm volatile("bar.sync 1, 160;" ::: "memory");
        }
      }
      __syncthreads();
      bad = *sm.flag;
      if (bad) break;  // identical decision in every CTA; no remote stores pending
      // (b') own diagonal rows take L11; own rows below form L21 = A21 L11^-T
      //      as one product, P[t][i] = sum_{s <= t} A21[i][s] Xi[t][s] (one
      //      output per thread, a chain of t + 1 FMAs), into the panel buffer;
      //      then the solved rows go back to W and to every other CTA.
      for (int e = tid; e < jb * jb; e += CHOL_THREADS) {
        const int u = e / jb, t = e % jb, i = j0 + u;
        if (i % NC == rank && t <= u) sm.W[(size_t)(i / NC) * k + j0 + t] = sm.D[u * B + t];
      }
      const int first = j0 + jb;
      int li0 = (first - rank + NC - 1) / NC;
      if (li0 < 0) li0 = 0;
      const int nrows = nloc - li0;
      T* P = sm.P[buf];
      for (int e = tid; e < nrows * jb; e += CHOL_THREADS) {
        const int lr = li0 + e / jb, t = e % jb, i = lr * NC + rank;
        if (i >= k) continue;
        const T* a = sm.W + (size_t)lr * k + j0;
        const T* xr = sm.Xi + t * B;
        T acc = T(0);
        for (int q = 0; q <= t; ++q) acc = fma(a[q], xr[q], acc);
        P[(size_t)t * k + i] = acc;
      }
      __syncthreads();
      for (int e = tid; e < nrows * jb; e += CHOL_THREADS) {
        const int lr = li0 + e / jb, t = e % jb, i = lr * NC + rank;
        if (i >= k) continue;
        const T x = P[(size_t)t * k + i];
        sm.W[(size_t)lr * k + j0 + t] = x;
        for (int q = 0; q < NC; ++q)
          if (q != rank) cluster.map_shared_rank(P, q)[(size_t)t * k + i] = x;
      }
      cluster.sync();
      // (c) trailing update of own rows: W[i][j] -= sum_t L21[i][t] L21[j][t],
      //     first <= j <= i; warp per row, lanes over j (P reads conflict-free).
      for (int lr = li0 + (tid >> 5); lr < nloc; lr += CHOL_THREADS / 32) {
        const int i = lr * NC + rank;
        if (i >= k) continue;
        T* wrow = sm.W + (size_t)lr * k;
        for (int j = first + (tid & 31); j <= i; j += 32) {
          T acc = T(0);
          for (int t = 0; t < jb; ++t) acc = fma(P[(size_t)t * k + i], P[(size_t)t * k + j], acc);
          wrow[j] -= acc;
        }
      }
      __syncthreads();
      buf ^= 1;
    }
    cluster.sync();
    if (!bad) {
      if (*sm.clamped && rank == 0 && tid == 0) raise_flag(flags, KFAC_FLAG_CHOL_SHIFTED);
      if (shift_out && rank == 0 && tid == 0) *shift_out = shift;
      ok = 1;
      break;
    }
  }

  if (!ok) {
    if (rank == 0 && tid == 0) {
      raise_flag(flags, finite_in ? KFAC_FLAG_CHOL_FAILED : (zero_in ? KFAC_FLAG_CHOL_SHIFTED : KFAC_FLAG_NONFINITE));
      if (shift_out) *shift_out = zero_in ? 1.0 : 0.0;
    }
    // Keep downstream finite: L = diag(sqrt(G_ii)), 1 where G_ii is not
    // positive and finite (L = I for the zero matrix).
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

size_t chol_smem_bytes(int k, int nloc, int B, size_t elt) {
  return elt * ((size_t)nloc * k + 2 * (size_t)B * B + B + 2 * (size_t)k * B) + 16;
}

// Cluster size nc_pref > 0 asks for that many CTAs (raised to the fewest whose
// shared memory holds the rows); 0 = one CTA per 16 rows, at most 16.
template <typename T>
cudaError_t launch_chol(const double* G, int k, double shift_rel, float* L32, int* flags,
                        unsigned long long* stats, cudaStream_t s, double* shift_out, int nc_pref, int panel) {
  {
    cudaError_t e = set_kernel_attrs_once(reinterpret_cast<const void*>(k_chol_cluster<T>), kSmemOptin, true);
    if (e != cudaSuccess) return e;
  }
  int nc = nc_pref > 0 ? nc_pref : (k + 15) / 16;
  if (nc > 16) nc = 16;
  if (nc < 1) nc = 1;
  int B = 16, nloc = 0;
  size_t smem = 0;
  const int B0 = panel == 32 ? 32 : 16;
  for (;; ++nc) {  // fewest CTAs from nc up whose rows fit (panel width B0, else halved down to 4)
    nloc = (k + nc - 1) / nc;
    for (B = B0; B >= 4; B /= 2) {
      smem = chol_smem_bytes(k, nloc, B, sizeof(T));
      if (smem <= (size_t)kSmemOptin) break;
    }
    if (smem <= (size_t)kSmemOptin || nc >= 16) break;
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
  return cudaLaunchKernelEx(&cfg, k_chol_cluster<T>, G, k, B, nloc, shift_rel, L32, flags, stats, shift_out);
}

// ---------------------------------------------------------------------------
// FP32 Cholesky of (G + shift I) on one CTA with the whole matrix in shared
// memory (k <= CTA_KMAX), for the CholeskyQR passes and the eigensolver's
// factor: no cluster barriers or distributed-memory broadcasts, which dominate
// the cluster kernel at these sizes. Right-looking, PW-column panels with a
// look-ahead of one panel:
//   (1) panel rows below the diagonal block: L21 = A21 L11^-T as a product
//       with the explicit inverse of L11 (formed with the factor), 4 x 4
//       output tiles per thread;
//   (2) the rank-PW update of the next block column (rows below it included);
//   (3) warp 0 factors and inverts the next PW x PW diagonal block in
//       registers (pivot and columns by shuffles) while the other 15 warps
//       apply the rank-PW update to the rest of the trailing lower triangle.
// The diagonal block's pivot chain is the critical path of (3) and its cost
// grows with PW^2, while the number of phases grows as k / PW: 16-column
// panels balance the two at k ~ 230. The updates use 4 x 4 output tiles per
// thread, a warp covering 8 x 4 tiles so that its row reads fall in distinct
// banks (odd row stride). Pivot floor, raised pivots and restarts follow the
// cluster kernel.
constexpr int CTA_THREADS = 512;
constexpr int CTA_WARPS = CTA_THREADS / 32;
constexpr int CTA_KMAX = 236;
constexpr int PW = 16;          // panel width
constexpr int XI_LD = PW + 1;   // row stride of the diagonal-block inverse

__host__ __device__ inline int cta_ks(int k) { return k | 1; }  // odd row stride: rows hit distinct banks
// A (k x ks), rinv (PW), Xi (PW x XI_LD), flags.
__host__ __device__ inline size_t cta_smem_bytes(int k) {
  return sizeof(float) * ((size_t)k * cta_ks(k) + PW + PW * XI_LD) + 16;
}

// Warp 0: factor the diagonal block A[j0 .. j0+jb)^2 (jb <= PW) in place,
// reciprocal pivots to rinv, the inverse of the factor to Xi (Xi[j][c] =
// (L11^-1)_jc, lower). Lane r < PW holds row r of the block and row r of W,
// which starts as I and takes the same row operations as the factorisation
// (scale row t by 1/L_tt, subtract L_rt times row t from the rows below), so
// that it ends as L11^-1. Sets sflag[0] on a non-finite pivot, sflag[1] on a
// raised one.
__device__ __forceinline__ void cta_factor_diag(float* A, int ks, int j0, int jb, float* rinv, float* Xi,
                                                const double* G, int k, double shift, float pfloor, int* sflag,
                                                int lane, int goff = 0) {
  float x[PW], w[PW];
  const int r = lane;
#pragma unroll
  for (int c = 0; c < PW; ++c) {
    x[c] = (r < jb && c < jb) ? (c <= r ? A[(size_t)(j0 + r) * ks + j0 + c] : 0.0f) : (r == c ? 1.0f : 0.0f);
    w[c] = (r == c) ? 1.0f : 0.0f;
  }
  // The replacement for a pivot below the floor, one FP64 operation per lane
  // up front (the FP64 pipe is slow, and the compiler may hoist the rare path).
  const float rp = r < jb ? raised_pivot(G, k, goff + j0 + r, shift, pfloor) : 1.0f;
  int bad = 0, clamped = 0;
#pragma unroll
  for (int t = 0; t < PW; ++t) {
    if (t >= jb) break;  // uniform: padded pivots are identity
    float piv = __shfl_sync(0xffffffffu, x[t], t);
    const float rpt = __shfl_sync(0xffffffffu, rp, t);
    if (!isfinite(piv)) bad = 1;
    else if (!(piv > pfloor)) {
      piv = rpt;
      clamped = 1;
    }
    const float y = rsqrt_newton(piv);
    if (r == t) {
      x[t] = piv * y;
      rinv[t] = y;
#pragma unroll
      for (int c = 0; c <= t; ++c) w[c] *= y;
    }
    const float lt = (r > t) ? x[t] * y : 0.0f;  // L[r][t]
    if (r > t) x[t] = lt;
#pragma unroll
    for (int c = t + 1; c < PW; ++c) {
      const float lc = __shfl_sync(0xffffffffu, lt, c);  // L[c][t]
      x[c] = fmaf(-lt, lc, x[c]);
    }
#pragma unroll
    for (int c = 0; c <= t; ++c) {
      const float wt = __shfl_sync(0xffffffffu, w[c], t);  // row t of L11^-1, final
      if (r > t) w[c] = fmaf(-lt, wt, w[c]);
    }
  }
  if (r < jb) {
#pragma unroll
    for (int c = 0; c < PW; ++c)
      if (c <= r) A[(size_t)(j0 + r) * ks + j0 + c] = x[c];
  }
  if (r < PW) {
#pragma unroll
    for (int c = 0; c < PW; ++c) Xi[r * XI_LD + c] = (r < jb && c <= r) ? w[c] : 0.0f;
  }
  bad = __any_sync(0xffffffffu, bad);
  clamped = __any_sync(0xffffffffu, clamped);
  if (lane == 0) { if (bad) sflag[0] = 1; if (clamped) sflag[1] = 1; }
}

// Rows [first, k) of the panel columns [j0, j0 + jb): L21 = A21 L11^-T, i.e.
// L21[i][c] = sum_s A21[i][s] Xi[c][s]. A warp owns (32 / CG) row groups x CG
// column groups of 4 x 4 outputs, CG = PW / 4 (at most one such task per
// warp for k <= CTA_KMAX); results are held in registers over a CTA barrier,
// then stored in place.
__device__ __forceinline__ void cta_panel_solve(float* A, int ks, int k, int j0, int jb, const float* Xi, int warp,
                                                int lane) {
  constexpr int CG = PW / 4, RG = 32 / CG;
  const int first = j0 + jb;
  const int i0 = first + 4 * RG * warp + 4 * (lane / CG), c0 = 4 * (lane % CG);
  const bool active = i0 < k && c0 < jb;
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
  if (active) {
    const float* pa[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) pa[u] = A + (size_t)min(i0 + u, k - 1) * ks + j0;
    for (int s2 = 0; s2 < jb; ++s2) {
      float av[4], xv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) av[u] = pa[u][s2];
#pragma unroll
      for (int v = 0; v < 4; ++v) xv[v] = Xi[(c0 + v) * XI_LD + s2];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], xv[v], acc[u][v]);
    }
  }
  __syncthreads();  // every read of A21 done before any store
  if (active) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if (i0 + u < k && c0 + v < jb) A[(size_t)(i0 + u) * ks + j0 + c0 + v] = acc[u][v];
  }
}

// A[i][c] -= sum_t A[i][j0+t] A[c][j0+t] for i in [r0, r1), c in [cb, c1),
// c <= i, t < jb (cb <= r0). Warps [w0, w0 + nw); each warp takes groups of
// 8 x 4 tiles (32 rows x 16 columns), a lane one 4 x 4 tile.
__device__ __forceinline__ void cta_rank_update(float* A, int ks, int k, int j0, int jb, int r0, int r1, int cb,
                                                int c1, int w0, int nw, int warp, int lane) {
  if (warp < w0 || r1 <= r0 || c1 <= cb) return;
  const int GR = (r1 - r0 + 31) / 32, GC = (c1 - cb + 15) / 16;
  // groups of row band gr that reach the diagonal: cb + 16 gc <= r0 + 32 gr + 31
  auto per_row = [&](int gr) { return min(GC, (r0 - cb + 32 * gr + 31) / 16 + 1); };
  int ngroups = 0;
  for (int gr = 0; gr < GR; ++gr) ngroups += per_row(gr);
  for (int grp = warp - w0; grp < ngroups; grp += nw) {
    int gr = 0, rem = grp;
    while (rem >= per_row(gr)) { rem -= per_row(gr); ++gr; }
    const int i0 = r0 + 32 * gr + 4 * (lane >> 2), c0 = cb + 16 * rem + 4 * (lane & 3);
    if (i0 >= r1 || c0 >= c1 || c0 > i0 + 3) continue;
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
    const float* pi[4];
    const float* pc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      pi[u] = A + (size_t)min(i0 + u, k - 1) * ks + j0;
      pc[u] = A + (size_t)min(c0 + u, k - 1) * ks + j0;
    }
    for (int t = 0; t < jb; ++t) {
      float ri[4], rcv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { ri[u] = pi[u][t]; rcv[u] = pc[u][t]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(ri[u], rcv[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int i = i0 + u, c = c0 + v;
        if (i < r1 && c < c1 && c <= i) A[(size_t)i * ks + c] -= acc[u][v];
      }
  }
}

// Block mode (blk.scal non-null): the kernel factors one diagonal block
// (k x k, rows and columns goff..goff+k of a kfull x kfull matrix) of a
// blocked factorisation. G32 is the block of the working matrix, already
// shifted and updated by the previous blocks; trace, shift and pivot floor come
// from blk.scal (the whole matrix's); raised pivots read the whole G's
// diagonal. With blk.retry, a non-finite pivot retries the block with a
// growing shift of its own diagonal (the blocked factorisation then factors
// G + shift I plus a block-diagonal extra shift: R stays invertible and
// span(Y R^-1) = span(Y), all a CholeskyQR pass needs); if every attempt
// fails, *blk.fail is set. L (k x k, row stride blk.ldl) is
// written without stats or shift_out.
struct CtaBlock {
  const double* scal;  // [trace, shift, pivot floor] of the whole matrix, or null
  int goff, kfull;
  int* fail;
  long long ldl;
  int retry;  // a block that overflows may be refactored with a shift of its own
};

__global__ void __launch_bounds__(CTA_THREADS, 1) k_chol_cta_f32(const double* __restrict__ G,
                                                                const float* __restrict__ G32, long long ld32,
                                                                int k, double shift_rel, float* __restrict__ L32,
                                                                int* flags, unsigned long long* stats,
                                                                double* shift_out, CtaBlock blk) {
  extern __shared__ __align__(16) float csm[];
  const bool block_mode = blk.scal != nullptr;
  if (block_mode && *blk.fail) return;  // an earlier block (or the input) failed: the finish step writes L
  const int ks = cta_ks(k);
  float* A = csm;                        // k x ks, row-major, lower part used
  float* rinv = A + (size_t)k * ks;      // PW reciprocal pivots of the current diagonal block
  float* Xi = rinv + PW;                 // PW x XI_LD: inverse of the current diagonal block
  int* sflag = reinterpret_cast<int*>(Xi + PW * XI_LD);  // [0] non-finite, [1] clamped
  __shared__ double s_trace;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (block_mode) {
    if (tid == 0) s_trace = blk.scal[0];
  } else if (warp == 0) {  // fixed-order trace
    double t = 0.0;
    for (int i = lane; i < k; i += 32) t += fabs(G[(size_t)i * k + i]);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) s_trace = t;
  }
  __syncthreads();
  const double trace = s_trace;
  const int kg = block_mode ? blk.kfull : k;  // order of the whole matrix (floor, raised pivots)
  const int goff = block_mode ? blk.goff : 0;
  // trace: sum of |G_ii| (the trace of a PSD matrix; a scale for the shifts and
  // the floor of any symmetric one). A zero diagonal means the zero matrix
  // (the Gram of a zero sketch, or a zero projected matrix): it is factored
  // exactly as G + 1 I = I I^T (L = I, shift 1).
  const bool finite_in = isfinite(trace) && trace > 0.0;
  const bool zero_in = trace == 0.0;
  const float pfloor = block_mode ? (float)blk.scal[2] : (float)fmax(1e-9 * trace, 1e-6 * trace / k);
  double shift = block_mode ? blk.scal[1]
                            : (shift_rel > 0.0 ? shift_rel * trace : (shift_rel < 0.0 ? -shift_rel * trace / k : 0.0));
  int ok = 0;
  const int attempts = (block_mode && !blk.retry) ? 1 : CHOL_ATTEMPTS;
  for (int attempt = 0; attempt < attempts && finite_in; ++attempt) {
    if (attempt > 0) {
      shift = fmax(shift, 1e-7 * trace) * 100.0;
      if (tid == 0) {
        raise_flag(flags, KFAC_FLAG_CHOL_SHIFTED);
        if (stats) atomicAdd(stats + STAT_CHOL_RETRY, 1ull);
      }
    }
    // a block of the working matrix carries the whole matrix's shift already:
    // only a retry's increase is added to its diagonal
    const float shf = block_mode ? (float)(shift - blk.scal[1]) : (float)shift;
    if (G32) {  // lower triangle by asynchronous copies (no registers, all in flight), then the shift
      for (int i = warp; i < k; i += CTA_WARPS) {
#pragma unroll 1
        for (int j = lane; j <= i; j += 32) cp_async4(A + (size_t)i * ks + j, G32 + (long long)i * ld32 + j, true);
      }
      cp_async_wait_all();
      __syncthreads();
      if (tid < k) A[(size_t)tid * ks + tid] += shf;
    } else {  // FP64 input (no FP32 copy given): converted element by element
      for (int i = warp; i < k; i += CTA_WARPS)
        for (int j = lane; j <= i; j += 32) A[(size_t)i * ks + j] = (float)G[(size_t)i * k + j] + (i == j ? shf : 0.0f);
    }
    if (tid == 0) { sflag[0] = 0; sflag[1] = 0; }
    __syncthreads();
    if (warp == 0) cta_factor_diag(A, ks, 0, min(PW, k), rinv, Xi, G, kg, shift, pfloor, sflag, lane, goff);
    __syncthreads();
    for (int j0 = 0; j0 < k && !sflag[0]; j0 += PW) {
      const int jb = min(PW, k - j0);
      const int first = j0 + jb;
      if (first >= k) break;
      const int jb1 = min(PW, k - first);
      cta_panel_solve(A, ks, k, j0, jb, Xi, warp, lane);
      __syncthreads();
      // Warp 1 applies the panel to the next diagonal block and releases warp 0
      // (named barrier 1), which factors it; meanwhile warps 1-15 update every
      // row below it, from the next block column to the diagonal.
      if (warp == 0) {
        asm volatile("bar.sync 1, %0;" ::"n"(CTA_THREADS) : "memory");
        cta_factor_diag(A, ks, first, jb1, rinv, Xi, G, kg, shift, pfloor, sflag, lane, goff);
      } else {
        cta_rank_update(A, ks, k, j0, jb, first, first + jb1, first, first + jb1, 1, 1, warp, lane);
        asm volatile("bar.arrive 1, %0;" ::"n"(CTA_THREADS) : "memory");
        cta_rank_update(A, ks, k, j0, jb, first + jb1, k, first, k, 1, CTA_WARPS - 1, warp, lane);
      }
      __syncthreads();
    }
    if (!sflag[0]) {
      if (tid == 0) {
        if (sflag[1]) raise_flag(flags, KFAC_FLAG_CHOL_SHIFTED);
        if (shift_out && !block_mode) *shift_out = shift;
      }
      ok = 1;
      break;
    }
    __syncthreads();
  }
  if (block_mode) {
    if (!ok) {
      if (tid == 0) *blk.fail = 1;
      return;
    }
    for (int i = warp; i < k; i += CTA_WARPS)
      for (int j = lane; j < k; j += 32) L32[(size_t)i * blk.ldl + j] = (j <= i) ? A[(size_t)i * ks + j] : 0.0f;
    return;
  }
  if (!ok) {
    if (tid == 0) {
      raise_flag(flags, finite_in ? KFAC_FLAG_CHOL_FAILED : (zero_in ? KFAC_FLAG_CHOL_SHIFTED : KFAC_FLAG_NONFINITE));
      if (shift_out) *shift_out = zero_in ? 1.0 : 0.0;
    }
    for (int i = warp; i < k; i += CTA_WARPS) {
      const double g = G[(size_t)i * k + i];
      for (int j = lane; j < k; j += 32)
        L32[(size_t)i * k + j] = (i == j) ? (float)sqrt(isfinite(g) && g > 1e-30 ? g : 1.0) : 0.0f;
    }
  } else {
    for (int i = warp; i < k; i += CTA_WARPS) {
#pragma unroll 4
      for (int j = lane; j < k; j += 32) L32[(size_t)i * k + j] = (j <= i) ? A[(size_t)i * ks + j] : 0.0f;
    }
  }
  if (stats && tid == 0) atomicAdd(stats + STAT_CHOL, 1ull);
}

}  // namespace

cudaError_t chol_cluster(const double* G, int k, double shift_rel, bool fp64, float* L32, int* flags,
                         unsigned long long* stats, cudaStream_t s, double* shift_out, const float* G32,
                         long long ld32, int nc_pref, int panel) {
  if (k <= 0) return cudaSuccess;
  if (!fp64 && k <= CTA_KMAX && cta_smem_bytes(k) <= (size_t)kSmemOptin) {
    cudaError_t e = set_kernel_attrs_once(reinterpret_cast<const void*>(k_chol_cta_f32), kSmemOptin, false);
    if (e != cudaSuccess) return e;
    k_chol_cta_f32<<<1, CTA_THREADS, cta_smem_bytes(k), s>>>(G, G32, ld32, k, shift_rel, L32, flags, stats,
                                                               shift_out, CtaBlock{});
    note_launch();
    return cudaGetLastError();
  }
  return fp64 ? launch_chol<double>(G, k, shift_rel, L32, flags, stats, s, shift_out, nc_pref, panel)
              : launch_chol<float>(G, k, shift_rel, L32, flags, stats, s, shift_out, nc_pref, panel);
}

// ---------------------------------------------------------------------------
// Blocked FP32 Cholesky for k > CTA_KMAX: right-looking over nb diagonal
// blocks of at most CTA_KMAX rows (sizes multiples of 4, so every block starts
// on a 16-byte boundary of the working matrix W = G + shift I):
//   L_bb = chol(W_bb)                        one-CTA kernel, block mode
//   L_rb^T = L_bb^-1 W_br                     the triangular solve below
//   W_rr <- W_rr - L_rb L_rb^T                symmetric tensor-core product (3xTF32)
// The pivots are those of the unblocked factorisation (up to rounding), so the
// floor, the raised pivots and the shift follow the one-CTA kernel; a
// non-finite pivot, or a zero or non-finite input, ends in the finish step's
// fallback factor as the other kernels' failure paths do.
namespace {
struct CbLayout {
  size_t scal, W, Lb, Xb, Xt, dinv, total;
  int nb, kb;
  long long kp, np, kbp;
};

CbLayout cb_layout(int k) {
  CbLayout c = {};
  c.nb = (k + CTA_KMAX - 1) / CTA_KMAX;
  for (;; ++c.nb) {
    c.kb = ((k + c.nb - 1) / c.nb + 3) / 4 * 4;
    if (c.kb <= CTA_KMAX) break;
  }
  c.kp = (k + 3) / 4 * 4;
  c.np = c.kp;
  c.kbp = c.kb;  // a multiple of 4
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = (off + 255) & ~size_t(255);
    off = o + bytes;
    return o;
  };
  c.scal = take(64);
  c.W = take(sizeof(float) * (size_t)k * c.kp);
  c.Lb = take(sizeof(float) * (size_t)c.kb * c.kb);
  c.Xb = take(sizeof(float) * (size_t)c.kb * c.np);
  c.Xt = take(sizeof(float) * (size_t)k * c.kbp);
  c.dinv = take(sizeof(float) * trsm_ws_floats(c.kb));
  c.total = off;
  return c;
}

// Trace, shift and pivot floor of the whole matrix (as the one-CTA kernel
// forms them), the failure marker (2: zero input, 3: non-finite input).
__global__ void k_cb_prep(const double* __restrict__ G, int k, double shift_rel, double* scal, int* fail) {
  const int lane = threadIdx.x;
  double t = 0.0;
  for (int i = lane; i < k; i += 32) t += fabs(G[(size_t)i * k + i]);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) {
    scal[0] = t;
    scal[1] = shift_rel > 0.0 ? shift_rel * t : (shift_rel < 0.0 ? -shift_rel * t / k : 0.0);
    scal[2] = (double)(float)fmax(1e-9 * t, 1e-6 * t / k);
    *fail = (t == 0.0) ? 2 : (isfinite(t) ? 0 : 3);
  }
}

// W = G32 + shift I (whole symmetric matrix, row stride kp), L32 = 0.
__global__ void k_cb_init(const float* __restrict__ G32, long long ld32, int k, const double* scal, float* W,
                          long long kp, float* L32) {
  const long long n = (long long)k * k;
  const float shf = (float)scal[1];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), j = (int)(e - (long long)i * k);
    W[(size_t)i * kp + j] = G32[(size_t)i * ld32 + j] + (i == j ? shf : 0.0f);
    L32[e] = 0.0f;
  }
}

// dst[r][c] = src[r][c] for r < rows, c < cols (dst row stride ldd).
__global__ void k_cb_place(const float* __restrict__ src, long long lds, int rows, int cols, float* dst,
                           long long ldd) {
  const long long n = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), c = (int)(e - (long long)r * cols);
    dst[(size_t)r * ldd + c] = src[(size_t)r * lds + c];
  }
}

// Flags, statistics and shift_out of the blocked factorisation; on failure the
// fallback factor diag(sqrt(G_ii)) (1 where G_ii is not positive and finite;
// I for the zero matrix) replaces L.
__global__ void k_cb_finish(const double* __restrict__ G, int k, const double* scal, const int* fail, float* L32,
                            int* flags, unsigned long long* stats, double* shift_out) {
  const int f = *fail;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (f) raise_flag(flags, f == 2 ? KFAC_FLAG_CHOL_SHIFTED : (f == 3 ? KFAC_FLAG_NONFINITE : KFAC_FLAG_CHOL_FAILED));
    if (shift_out) *shift_out = f == 0 ? scal[1] : (f == 2 ? 1.0 : 0.0);
    if (stats) atomicAdd(stats + STAT_CHOL, 1ull);
  }
  if (!f) return;
  const long long n = (long long)k * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), j = (int)(e - (long long)i * k);
    const double g = G[(size_t)i * k + i];
    L32[e] = (i == j) ? (float)sqrt(isfinite(g) && g > 1e-30 ? g : 1.0) : 0.0f;
  }
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>(1216, (n + 255) / 256)); }
}  // namespace

size_t chol_blocked_ws_bytes(int k) { return k > CTA_KMAX ? cb_layout(k).total : 0; }

namespace {
__global__ void k_factor_unscale(float* __restrict__ L32, int k, const double* __restrict__ dscale) {
  const long long n = (long long)k * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / k);
    L32[e] = (float)((double)L32[e] * dscale[i]);
  }
}
}  // namespace

cudaError_t factor_unscale(float* L32, int k, const double* dscale, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_factor_unscale<<<grid_for((long long)k * k), 256, 0, s>>>(L32, k, dscale);
  note_launch();
  return cudaGetLastError();
}

cudaError_t chol_blocked(const double* G, const float* G32, long long ld32, int k, double shift_rel, float* L32,
                         int* flags, unsigned long long* stats, cudaStream_t s, double* shift_out, void* ws,
                         long long wait_cycles) {
  if (k <= CTA_KMAX) return chol_cluster(G, k, shift_rel, false, L32, flags, stats, s, shift_out, G32, ld32);
  const CbLayout c = cb_layout(k);
  char* base = static_cast<char*>(ws);
  double* scal = reinterpret_cast<double*>(base + c.scal);
  int* fail = reinterpret_cast<int*>(scal + 4);
  float* W = reinterpret_cast<float*>(base + c.W);
  float* Lb = reinterpret_cast<float*>(base + c.Lb);
  float* Xb = reinterpret_cast<float*>(base + c.Xb);
  float* Xt = reinterpret_cast<float*>(base + c.Xt);
  float* dinv = reinterpret_cast<float*>(base + c.dinv);
  {
    cudaError_t e = set_kernel_attrs_once(reinterpret_cast<const void*>(k_chol_cta_f32), kSmemOptin, false);
    if (e != cudaSuccess) return e;
  }
  k_cb_prep<<<1, 32, 0, s>>>(G, k, shift_rel, scal, fail);
  note_launch();
  k_cb_init<<<grid_for((long long)k * k), 256, 0, s>>>(G32, ld32, k, scal, W, c.kp, L32);
  note_launch();
  for (int o = 0; o < k; o += c.kb) {
    const int kb = std::min(c.kb, k - o), n = k - o - kb;
    float* Wbb = W + (size_t)o * c.kp + o;
    // shift_out asks for one shift of the whole matrix (the eigensolver
    // subtracts it): no block may add its own
    CtaBlock blk{scal, o, k, fail, kb, shift_out ? 0 : 1};
    k_chol_cta_f32<<<1, CTA_THREADS, cta_smem_bytes(kb), s>>>(G, Wbb, c.kp, kb, 0.0, Lb, flags, nullptr, nullptr,
                                                                blk);
    note_launch();
    k_cb_place<<<grid_for((long long)kb * kb), 256, 0, s>>>(Lb, kb, kb, kb, L32 + (size_t)o * k + o, k);
    note_launch();
    if (n == 0) break;
    cudaError_t e = trsm_lower_f32(Lb, kb, Wbb + kb, c.kp, Xb, c.np, n, dinv, s);  // L_rb^T (kb x n)
    if (e != cudaSuccess) return e;
    if ((e = transpose_f32(Xb, c.np, kb, n, Xt, c.kbp, s)) != cudaSuccess) return e;  // L_rb (n x kb)
    k_cb_place<<<grid_for((long long)n * kb), 256, 0, s>>>(Xt, c.kbp, n, kb, L32 + (size_t)(o + kb) * k + o, k);
    note_launch();
    float* Wrr = W + (size_t)(o + kb) * c.kp + o + kb;
    if ((e = syrk_update(s, n, kb, Xt, (int)c.kbp, -1.0f, 1.0f, KFAC_PREC_FP32, Wrr, (int)c.kp, flags,
                         wait_cycles)) != cudaSuccess)
      return e;
  }
  k_cb_finish<<<grid_for((long long)k * k), 256, 0, s>>>(G, k, scal, fail, L32, flags, stats, shift_out);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Qt = L^-1 Yt with the FP32 lower factor, for all d columns of Yt at once.
// The inverses of L's 32 x 32 diagonal blocks are formed first (one warp per
// block, one lane per column); each CTA then owns 32 columns of Yt, keeps its
// k x 32 slab of the solution in shared memory and, row block by row block,
// subtracts the solved blocks (L_IJ X_J through 32 x 32 tiles of L) and applies
// the block inverse: all multiply-adds, no sequential per-row solve.
namespace {
constexpr int TR_COLS = 32, TR_RB = 32, TR_THREADS = 256;

__global__ void __launch_bounds__(32) k_diag_block_inv(const float* __restrict__ L, int k, float* __restrict__ Dinv) {
  __shared__ float Lb[TR_RB][TR_RB + 1];
  const int blk = blockIdx.x, i0 = blk * TR_RB, ib = min(TR_RB, k - i0), c = threadIdx.x;
  float lv[TR_RB];  // all 32 loads in flight (one at a time each waits out the L2 latency)
#pragma unroll
  for (int a = 0; a < TR_RB; ++a) lv[a] = (a < ib && c < ib) ? L[(size_t)(i0 + a) * k + i0 + c] : (a == c ? 1.f : 0.f);
#pragma unroll
  for (int a = 0; a < TR_RB; ++a) Lb[a][c] = lv[a];
  __syncwarp();
  float x[TR_RB];  // column c of the block inverse
#pragma unroll
  for (int i = 0; i < TR_RB; ++i) {
    float v = (i == c) ? 1.0f : 0.0f;
#pragma unroll
    for (int u = 0; u < i; ++u) v = fmaf(-Lb[i][u], x[u], v);
    x[i] = (i >= c) ? v * __frcp_rn(Lb[i][i]) : 0.0f;  // correctly rounded reciprocal, no divide slow path
  }
  float* out = Dinv + (size_t)blk * TR_RB * TR_RB;
#pragma unroll
  for (int i = 0; i < TR_RB; ++i) out[i * TR_RB + c] = x[i];
}

// The tiles of L this CTA multiplies by arrive through a two-slot ring of
// cp.async copies issued one tile ahead: tile s of the sequence L(I, 0), ...,
// L(I, I-1), Dinv(I) over the block rows I (s = I (I+1) / 2 + M) is copied
// while tile s - 1 is used, so the loop waits on L2 once per block row of the
// ring instead of once per tile.
__device__ __forceinline__ void trsm_tile_async(float* dst, const float* __restrict__ L, const float* __restrict__ Dinv,
                                                int k, int I, int M, int tid) {
  const int i0 = I * TR_RB, ib = min(TR_RB, k - i0);
  if (M < I) {  // off-diagonal tile of L: rows i0.., columns 32 M..
    for (int e = tid; e < TR_RB * TR_RB; e += TR_THREADS) {
      const int a = e / TR_RB, b = e % TR_RB;
      const bool ok = a < ib;
      cp_async4(dst + a * (TR_RB + 1) + b, L + (ok ? (size_t)(i0 + a) * k + (size_t)TR_RB * M + b : 0), ok);
    }
  } else {      // the block inverse of the diagonal block
    const float* Di = Dinv + (size_t)I * TR_RB * TR_RB;
    for (int e = tid; e < TR_RB * TR_RB; e += TR_THREADS)
      cp_async4(dst + (e / TR_RB) * (TR_RB + 1) + e % TR_RB, Di + e, true);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__global__ void __launch_bounds__(TR_THREADS) k_trsm_lower(const float* __restrict__ L, const float* __restrict__ Dinv,
                                                            int k, const float* __restrict__ Yt, long long ldy,
                                                            float* __restrict__ Qt, long long ldq, int d,
                                                            float* __restrict__ Qlo, long long ldlo) {
  extern __shared__ __align__(16) float tsm[];
  float* X = tsm;                          // kpad x TR_COLS
  const int kpad = (k + TR_RB - 1) / TR_RB * TR_RB;
  const int T = kpad / TR_RB;
  float* ring = X + (size_t)kpad * TR_COLS;  // 2 x TR_RB x (TR_RB + 1)
  constexpr int TILE = TR_RB * (TR_RB + 1);
  const int tid = threadIdx.x, c = tid & 31, r0 = tid >> 5;  // 8 row groups
  const int col0 = blockIdx.x * TR_COLS;
  const int col = col0 + c;
  int s = 0;                                // tile sequence index of the tile in use
  trsm_tile_async(ring, L, Dinv, k, 0, 0, tid);
  for (int I = 0; I < T; ++I) {
    const int i0 = I * TR_RB, ib = min(TR_RB, k - i0);
    float acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int ri = r0 + 8 * u;
      acc[u] = (ri < ib && col < d) ? Yt[(long long)(i0 + ri) * ldy + col] : 0.0f;
    }
    for (int M = 0; M <= I; ++M, ++s) {
      // prefetch the next tile of the sequence into the other slot, then wait for this one
      const int nI = (M < I) ? I : I + 1, nM = (M < I) ? M + 1 : 0;
      if (nI < T) {
        trsm_tile_async(ring + ((s + 1) & 1) * TILE, L, Dinv, k, nI, nM, tid);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
      __syncthreads();
      const float* Lt = ring + (s & 1) * TILE;
      if (M < I) {  // acc -= L(I, M) X_M
#pragma unroll 8
        for (int mm = 0; mm < TR_RB; ++mm) {
          float x = X[(size_t)(TR_RB * M + mm) * TR_COLS + c];
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u] = fmaf(-Lt[(r0 + 8 * u) * (TR_RB + 1) + mm], x, acc[u]);
        }
      } else {      // X_I = Dinv_I * acc: stage acc, then multiply by the block inverse
#pragma unroll
        for (int u = 0; u < 4; ++u) X[(size_t)(i0 + r0 + 8 * u) * TR_COLS + c] = (r0 + 8 * u < ib) ? acc[u] : 0.0f;
        __syncthreads();
        float out[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
        for (int u = 0; u < TR_RB; ++u) {
          const float x = X[(size_t)(i0 + u) * TR_COLS + c];
#pragma unroll
          for (int v = 0; v < 4; ++v) out[v] = fmaf(Lt[(r0 + 8 * v) * (TR_RB + 1) + u], x, out[v]);
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int ri = r0 + 8 * v;
          if (ri < ib) {
            X[(size_t)(i0 + ri) * TR_COLS + c] = out[v];
            if (col < d) {
              Qt[(long long)(i0 + ri) * ldq + col] = out[v];
              if (Qlo) Qlo[(long long)(i0 + ri) * ldlo + col] = tf32_tail(out[v]);
            }
          }
        }
      }
      __syncthreads();  // the slot just used is refilled by the next iteration's prefetch
    }
  }
}
// Packs L for k_trsm_lower_smem once per solve (instead of every CTA
// gathering it with 4-byte copies): block row I of 32 rows at offset
// 1024 I (I+1) / 2 with row width 32 (I+1), the off-diagonal blocks copied
// from L and the diagonal block replaced by its inverse (warp 0, as
// k_diag_block_inv). One CTA per block row.
__global__ void __launch_bounds__(256) k_trsm_pack(const float* __restrict__ L, int k, float* __restrict__ Lp) {
  __shared__ float Lb[TR_RB][TR_RB + 1];
  const int I = blockIdx.x, i0 = I * TR_RB, ib = min(TR_RB, k - i0), tid = threadIdx.x;
  const int width = 32 * (I + 1);
  float* dst = Lp + (size_t)512 * I * (I + 1);
  // off-diagonal part, eight loads in flight per thread
  const int tot = 32 * 32 * I;
  for (int e0 = 0; e0 < tot; e0 += 8 * 256) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = e0 + q * 256 + tid, a = e / (32 * I), cc = e - a * 32 * I;
      v[q] = (e < tot && a < ib) ? L[(size_t)(i0 + a) * k + cc] : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = e0 + q * 256 + tid, a = e / (32 * I), cc = e - a * 32 * I;
      if (e < tot) dst[(size_t)a * width + cc] = v[q];
    }
  }
  if (tid < 32) {  // diagonal block inverse, lane c = column c
    const int c = tid;
    float lv[TR_RB];
#pragma unroll
    for (int a = 0; a < TR_RB; ++a) lv[a] = (a < ib && c < ib) ? L[(size_t)(i0 + a) * k + i0 + c] : (a == c ? 1.f : 0.f);
#pragma unroll
    for (int a = 0; a < TR_RB; ++a) Lb[a][c] = lv[a];
    __syncwarp();
    float x[TR_RB];
#pragma unroll
    for (int i = 0; i < TR_RB; ++i) {
      float v = (i == c) ? 1.0f : 0.0f;
#pragma unroll
      for (int u = 0; u < i; ++u) v = fmaf(-Lb[i][u], x[u], v);
      x[i] = (i >= c) ? v * __frcp_rn(Lb[i][i]) : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < TR_RB; ++i) dst[(size_t)i * width + 32 * I + c] = x[i];
  }
}

// The same solve with the whole lower factor resident in shared memory (for
// k <= 32 * TS_MAXT): the 32-row block rows of L are packed once (their
// diagonal blocks replaced by the block inverses) and the CTA's 32 columns of
// Yt are kept column-major, so the block substitution runs from shared memory
// with 128-bit reads: per 4 steps of the inner product, one float4 of the
// column and one broadcast float4 of each of the thread's 4 rows of L.
constexpr int TS_MAXT = 9;

__host__ __device__ inline size_t trsm_smem_floats(int T) {
  return (size_t)1024 * T * (T + 1) / 2 + (size_t)32 * (32 * T + 4) + 32 * 33;
}

__global__ void __launch_bounds__(TR_THREADS) k_trsm_lower_smem(const float* __restrict__ Lpk, int k, int T,
                                                                 const float* __restrict__ Yt, long long ldy,
                                                                 float* __restrict__ Qt, long long ldq, int d,
                                                                 float* __restrict__ Qlo, long long ldlo) {
  extern __shared__ __align__(16) float tsm[];
  const int kpad = 32 * T, xs = kpad + 4;
  float* Lp = tsm;                                     // block row I at 1024 I (I+1) / 2: [32][32 (I+1)]
  float* Xc = Lp + (size_t)1024 * T * (T + 1) / 2;     // [32 columns][xs]: the solution, column-major
  float* Ts = Xc + (size_t)32 * xs;                    // [32][33]: one block of partial sums
  const int tid = threadIdx.x, c = tid & 31, w = tid >> 5;  // w: rows 4w..4w+3 of a block
  const int col0 = blockIdx.x * TR_COLS, col = col0 + c;
  {  // the packed factor (k_trsm_pack), 16 bytes per copy
    const int n4 = 128 * T * (T + 1);  // 512 T (T+1) floats
    for (int e = tid; e < n4; e += TR_THREADS) cp_async16(Lp + 4 * e, Lpk + 4 * e);
  }
  for (int i = w; i < kpad; i += TR_THREADS / 32) {  // warp per row of Yt, lanes over the 32 columns
    const bool ok = i < k && col < d;
    cp_async4(Xc + (size_t)c * xs + i, Yt + (ok ? (long long)i * ldy + col : 0), ok);
  }
  cp_async_wait_all();
  __syncthreads();
  const float* xcol = Xc + (size_t)c * xs;
  for (int I = 0; I < T; ++I) {
    const int width = 32 * (I + 1);
    const float* Lb = Lp + (size_t)512 * I * (I + 1);
    float acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = xcol[32 * I + 4 * w + u];
    for (int mm = 0; mm < 32 * I; mm += 4) {
      const float4 x = *reinterpret_cast<const float4*>(xcol + mm);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 l = *reinterpret_cast<const float4*>(Lb + (size_t)(4 * w + u) * width + mm);
        acc[u] = fmaf(-l.x, x.x, acc[u]);
        acc[u] = fmaf(-l.y, x.y, acc[u]);
        acc[u] = fmaf(-l.z, x.z, acc[u]);
        acc[u] = fmaf(-l.w, x.w, acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) Ts[c * 33 + 4 * w + u] = acc[u];
    __syncthreads();
    float out[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
    for (int v = 0; v < 32; ++v) {
      const float tv = Ts[c * 33 + v];
#pragma unroll
      for (int u = 0; u < 4; ++u) out[u] = fmaf(Lb[(size_t)(4 * w + u) * width + 32 * I + v], tv, out[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int row = 32 * I + 4 * w + u;
      Xc[(size_t)c * xs + row] = out[u];
      if (row < k && col < d) {
        Qt[(long long)row * ldq + col] = out[u];
        if (Qlo) Qlo[(long long)row * ldlo + col] = tf32_tail(out[u]);
      }
    }
    __syncthreads();
  }
}
}  // namespace

cudaError_t trsm_lower_f32(const float* L, int k, const float* Yt, long long ldy, float* Qt, long long ldq, int d,
                           float* dinv_ws, cudaStream_t s, float* qlo, long long ldlo) {
  if (k <= 0 || d <= 0) return cudaSuccess;
  const int kpad = (k + TR_RB - 1) / TR_RB * TR_RB;  // X rows incl. the padded tail block
  size_t smem = sizeof(float) * ((size_t)kpad * TR_COLS + 2 * TR_RB * (TR_RB + 1));
  if (smem > (size_t)kSmemOptin) return cudaErrorInvalidValue;
  {
    cudaError_t e = set_kernel_attrs_once(reinterpret_cast<const void*>(k_trsm_lower), kSmemOptin, false);
    if (e != cudaSuccess) return e;
  }
  const int T = kpad / TR_RB;
  if (T <= TS_MAXT) {
    cudaError_t e = set_kernel_attrs_once(reinterpret_cast<const void*>(k_trsm_lower_smem), kSmemOptin, false);
    if (e != cudaSuccess) return e;
    const size_t smem_all = sizeof(float) * trsm_smem_floats(T);
    if (smem_all <= (size_t)kSmemOptin) {
      k_trsm_pack<<<T, 256, 0, s>>>(L, k, dinv_ws);
      note_launch();
      k_trsm_lower_smem<<<(d + TR_COLS - 1) / TR_COLS, TR_THREADS, smem_all, s>>>(dinv_ws, k, T, Yt, ldy, Qt, ldq,
                                                                                  d, qlo, ldlo);
      note_launch();
      return cudaGetLastError();
    }
  }
  k_diag_block_inv<<<(k + TR_RB - 1) / TR_RB, 32, 0, s>>>(L, k, dinv_ws);
  note_launch();
  k_trsm_lower<<<(d + TR_COLS - 1) / TR_COLS, TR_THREADS, smem, s>>>(L, dinv_ws, k, Yt, ldy, Qt, ldq, d, qlo, ldlo);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Blocked triangular solve Qt = L^-1 Yt for k above the shared-memory solve's
// range, over the diagonal blocks of the blocked Cholesky (at most CTA_KMAX
// rows, multiples of 4). Block row I: the residual R_I = Y_I - L_I,<I X_<I is
// one FP32-accurate tensor-core product (A = L's rows of block I with a padded
// stride, B = the solved rows so far, kept transposed in XT: d x k), then
// X_I = L_II^-1 R_I by the shared-memory solve, then X_I is transposed into XT.
namespace {
struct TbLayout {
  size_t Lp, Lbb, dinv, XT, R, total;
  int kb;
  long long kp, ldr;
};

TbLayout tb_layout(int k, int d) {
  TbLayout t = {};
  const CbLayout c = cb_layout(k);
  t.kb = c.kb;
  t.kp = c.kp;
  t.ldr = (d + 3) / 4 * 4;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = (off + 255) & ~size_t(255);
    off = o + bytes;
    return o;
  };
  t.Lp = take(sizeof(float) * (size_t)k * t.kp);
  t.Lbb = take(sizeof(float) * (size_t)t.kb * t.kb);
  t.dinv = take(sizeof(float) * trsm_ws_floats(t.kb));
  t.XT = take(sizeof(float) * (size_t)d * t.kp);
  t.R = take(sizeof(float) * (size_t)t.kb * t.ldr);
  t.total = off;
  return t;
}
}  // namespace

bool trsm_blocked_used(int k) { return k > TS_MAXT * TR_RB; }

size_t trsm_blocked_ws_bytes(int k, int d) { return trsm_blocked_used(k) ? tb_layout(k, d).total : 0; }

cudaError_t trsm_blocked(const float* L, int k, const float* Yt, long long ldy, float* Qt, long long ldq, int d,
                         void* ws, int* flags, long long wait_cycles, cudaStream_t s) {
  if (k <= 0 || d <= 0) return cudaSuccess;
  const TbLayout t = tb_layout(k, d);
  char* base = static_cast<char*>(ws);
  float* Lp = reinterpret_cast<float*>(base + t.Lp);
  float* Lbb = reinterpret_cast<float*>(base + t.Lbb);
  float* dinv = reinterpret_cast<float*>(base + t.dinv);
  float* XT = reinterpret_cast<float*>(base + t.XT);
  float* R = reinterpret_cast<float*>(base + t.R);
  k_cb_place<<<grid_for((long long)k * k), 256, 0, s>>>(L, k, k, k, Lp, t.kp);
  note_launch();
  cudaError_t e;
  for (int o = 0; o < k; o += t.kb) {
    const int kb = std::min(t.kb, k - o);
    const float* src = Yt + (size_t)o * ldy;
    long long lds = ldy;
    if (o > 0) {  // R = Y_I - L_I,<I X_<I
      GemmDesc<float> g = {};
      g.M = kb; g.N = d; g.K = o;
      g.A = Lp + (size_t)o * t.kp; g.sam = t.kp; g.sak = 1;
      g.B = XT; g.sbn = t.kp; g.sbk = 1;
      g.D = R; g.ldd = t.ldr;
      g.C0 = Yt + (size_t)o * ldy; g.ldc = ldy;
      g.alpha = -1.0f; g.beta = 1.0f; g.zsplit = 1;
      g.flags = flags; g.wait_cycles = wait_cycles;
      if ((e = gemm_f32(g, KFAC_PREC_FP32, s)) != cudaSuccess) return e;
      src = R;
      lds = t.ldr;
    }
    k_cb_place<<<grid_for((long long)kb * kb), 256, 0, s>>>(Lp + (size_t)o * t.kp + o, t.kp, kb, kb, Lbb, kb);
    note_launch();
    if ((e = trsm_lower_f32(Lbb, kb, src, lds, Qt + (size_t)o * ldq, ldq, d, dinv, s)) != cudaSuccess) return e;
    if (o + kb < k && (e = transpose_f32(Qt + (size_t)o * ldq, ldq, kb, d, XT + o, t.kp, s)) != cudaSuccess)
      return e;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Qt = L^-1 Yt through the explicit inverse: Linv = L^-1 by the triangular
// solve of the k x k identity (the shared-memory or the blocked form), Y = Yt^T
// by a transpose, then one FP32-accurate tensor-core product Qt = (Y Linv^T)^T
// (both operands K-major, transposed store). The k x k inverse is small; the
// k^2 d product, which the substitution spends on the SIMT pipes, runs on the
// tensor cores.
namespace {
__global__ void k_identity(float* __restrict__ E, int k, long long ld) {
  const long long n = (long long)k * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / ld, j = e - i * ld;
    E[e] = (i == j) ? 1.0f : 0.0f;
  }
}

struct TiLayout {
  size_t E, Linv, Y, dinv, inner, total;
  long long kp;
};

TiLayout ti_layout(int k, int d) {
  TiLayout t = {};
  t.kp = (k + 3) / 4 * 4;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = (off + 255) & ~size_t(255);
    off = o + bytes;
    return o;
  };
  t.E = take(sizeof(float) * (size_t)k * t.kp);
  t.Linv = take(sizeof(float) * (size_t)k * t.kp);
  t.Y = take(sizeof(float) * (size_t)d * t.kp);
  t.dinv = take(sizeof(float) * trsm_ws_floats(k));
  t.inner = take(trsm_blocked_ws_bytes(k, k));
  t.total = off;
  return t;
}
}  // namespace

size_t trsm_inverse_ws_bytes(int k, int d) { return k > 0 && d > 0 ? ti_layout(k, d).total : 0; }

cudaError_t trsm_inverse(const float* L, int k, const float* Yt, long long ldy, float* Qt, long long ldq, int d,
                         void* ws, int* flags, long long wait_cycles, cudaStream_t s, const double* dscale) {
  if (k <= 0 || d <= 0) return cudaSuccess;
  const TiLayout t = ti_layout(k, d);
  char* base = static_cast<char*>(ws);
  float* E = reinterpret_cast<float*>(base + t.E);
  float* Linv = reinterpret_cast<float*>(base + t.Linv);
  float* Y = reinterpret_cast<float*>(base + t.Y);
  k_identity<<<grid_for((long long)k * t.kp), 256, 0, s>>>(E, k, t.kp);
  note_launch();
  cudaError_t e = trsm_blocked_used(k)
                      ? trsm_blocked(L, k, E, t.kp, Linv, t.kp, k, base + t.inner, flags, wait_cycles, s)
                      : trsm_lower_f32(L, k, E, t.kp, Linv, t.kp, k, reinterpret_cast<float*>(base + t.dinv), s);
  if (e != cudaSuccess) return e;
  if ((e = transpose_f32(Yt, ldy, k, d, Y, t.kp, s, dscale)) != cudaSuccess) return e;
  GemmDesc<float> g = {};
  g.M = d; g.N = k; g.K = k;
  g.A = Y; g.sam = t.kp; g.sak = 1;
  g.B = Linv; g.sbn = t.kp; g.sbk = 1;
  g.D = Qt; g.ldd = ldq; g.d_trans = 1;
  g.alpha = 1.0f; g.zsplit = 1;
  g.flags = flags; g.wait_cycles = wait_cycles;
  return gemm_f32(g, KFAC_PREC_FP32, s);
}

}  // namespace kfac
