// Eigensolver for the small projected matrix C = Q^T F Q ("Eigen_decomp" of
// Alg. 3), and for whole factors with d <= k.
//
//  1. eig_jacobi_f32: C + s I (s a small PD shift) is Cholesky-factored in FP32
//     on a cluster (C + s I = L L^T) and the columns of W = L are made mutually
//     orthogonal by one-sided (Hestenes) Jacobi rotations W <- W J. Since
//     W W^T = C + s I is invariant, at convergence the unit columns of W are
//     eigenvectors of C and |w_j|^2 - s its eigenvalues; only one k x k FP32
//     matrix is stored. The sweeps run on a thread-block cluster as a block
//     round-robin: one warp per column pair, one cluster barrier per
//     block-round.
//  2. eig_refine_f32 / eig_refine_f64: one refinement step of all eigenpairs
//     (Ogita and Aishima, "Iterative refinement for symmetric eigenvalue
//     decomposition", 2018): from R = I - X^T X and S = X^T C X,
//     lam_i = S_ii / (1 - R_ii) and X <- X + X E with
//     E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i) for separated pairs,
//     R_ij / 2 otherwise. The k x k products run in FP32 (default) or FP64,
//     spread over many CTAs; X and lam are carried in FP64.
//  3. eig_select: descending stable sort, leading r pairs, damping coefficients.
#include <algorithm>
#include <cooperative_groups.h>

#include "common.cuh"
#include "gemm.cuh"

namespace cg = cooperative_groups;

namespace kfac {
namespace {

// Threads per CTA: one warp per column pair of a block-round, so blocks of up
// to 8 columns run 8 warps (fewer idle warps at every barrier: 2-4% faster at
// k = 74 and 230), wider blocks 16.
constexpr int EIG_THREADS_MAX = 512;
constexpr int EIG_MAX_NC = 16;  // non-portable cluster size, enabled at launch

// Butterfly sum: every lane ends with the same total (each level adds the same
// two operands in every lane, and FP addition is commutative).
__device__ __forceinline__ float warp_sum_all(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of squares of a register column, the same total in every lane.
template <int NI>
__device__ __forceinline__ float col_sumsq(const float4 (&x)[NI]) {
  float s = 0.f;
#pragma unroll
  for (int it = 0; it < NI; ++it)
    s = fmaf(x[it].x, x[it].x, fmaf(x[it].y, x[it].y, fmaf(x[it].z, x[it].z, fmaf(x[it].w, x[it].w, s))));
  return warp_sum_all(s);
}

// Columns are zero-padded to NI * 128 floats: each lane holds NI float4s of a
// column (lane + 32 * it), and the padding stays zero under rotations.
template <int NI>
__device__ __forceinline__ void col_load(const float* sm, int off, float4 (&x)[NI], int lane) {
  const float4* p = reinterpret_cast<const float4*>(sm + off);
#pragma unroll
  for (int it = 0; it < NI; ++it) x[it] = p[lane + 32 * it];
}
template <int NI>
__device__ __forceinline__ void col_store(float* sm, int off, const float4 (&x)[NI], int lane) {
  float4* p = reinterpret_cast<float4*>(sm + off);
#pragma unroll
  for (int it = 0; it < NI; ++it) p[lane + 32 * it] = x[it];
}

// Rotate register columns x, y (squared norms al, be, warp-uniform) to make
// them orthogonal (one warp). Returns 1 if a rotation was applied; al and be
// then hold the new squared norms.
template <int NI>
__device__ __forceinline__ int jacobi_rot(float4 (&x)[NI], float4 (&y)[NI], float& al, float& be, float tol,
                                          float& off2) {
  float ga = 0.f;
#pragma unroll
  for (int it = 0; it < NI; ++it)
    ga = fmaf(x[it].x, y[it].x, fmaf(x[it].y, y[it].y, fmaf(x[it].z, y[it].z, fmaf(x[it].w, y[it].w, ga))));
  ga = warp_sum_all(ga);
  const float g2 = ga * ga, ab = al * be;
  if (ab > 0.0f) off2 = fmaxf(off2, __fdividef(g2, ab));  // squared cosine of the pair's angle
  if (!(ga != 0.0f && g2 > (tol * tol) * ab)) return 0;
  // 2x2 symmetric Schur step on the Gram [[al, ga], [ga, be]]: J = [[c, s], [-s, c]],
  // t = sign(z) / (|z| + sqrt(1 + z^2)), z = (be - al) / (2 ga): scale-invariant
  // (a form that squares be - al and ga underflows on factors of scale ~1e-6).
  // Fast reciprocal / rsqrt: their ulp errors only perturb the rotation slightly
  // (W W^T stays C + sI to FP32 accuracy) and the refinement absorbs them.
  const float zeta = __fdividef(be - al, 2.0f * ga);
  const float az = fabsf(zeta);
  float t;
  if (az > 1e15f) {
    t = __fdividef(0.5f, zeta);
  } else {
    const float q = fmaf(zeta, zeta, 1.0f);
    t = copysignf(__fdividef(1.0f, az + q * rsqrtf(q)), zeta);
  }
  const float cs = rsqrtf(fmaf(t, t, 1.0f)), sn = cs * t;
#pragma unroll
  for (int it = 0; it < NI; ++it) {
    const float4 a4 = x[it], b4 = y[it];
    x[it] = make_float4(cs * a4.x - sn * b4.x, cs * a4.y - sn * b4.y, cs * a4.z - sn * b4.z, cs * a4.w - sn * b4.w);
    y[it] = make_float4(sn * a4.x + cs * b4.x, sn * a4.y + cs * b4.y, sn * a4.z + cs * b4.z, sn * a4.w + cs * b4.w);
  }
  // t solves t^2 + 2 z t - 1 = 0, so the squared norms become al - t ga and
  // be + t ga (their sum is invariant). One of them shrinks; where it loses
  // more than half, the update would cancel and both are recomputed.
  float al2 = fmaf(-t, ga, al), be2 = fmaf(t, ga, be);
  if (!(al2 > 0.5f * al) || !(be2 > 0.5f * be)) {
    al2 = col_sumsq<NI>(x);
    be2 = col_sumsq<NI>(y);
  }
  al = al2;
  be = be2;
  return 1;
}

// Position p (0 <= p < m) of a round-robin tournament of m players at round r:
// player 0 never moves, the others rotate. Pairing position p with m-1-p over
// rounds r = 0..m-2 meets every pair of players exactly once.
__device__ __forceinline__ int rr_player(int p, int r, int m) {
  return p == 0 ? 0 : 1 + (p - 1 + r) % (m - 1);
}

struct EigArgs {
  const float* L;       // k x k lower factor of C + shift I, row-major FP32 (column j of W = column j of L)
  const double* shift;  // device scalar: the shift that factorisation used
  int k;
  int max_sweeps;
  float tol;
  double* X;
  double* lam;
  int* flags;
  unsigned long long* stats;
  int b;   // columns per block (the cluster holds 2 * NC blocks)
  int kp;  // padded column length in shared memory (multiple of 128)
  float stop_tol;  // > 0: stop after a sweep whose largest pair cosine was below it
  int full;        // 0: L is lower triangular (only i >= j is read); 1: a full matrix
};

// One-sided Jacobi on the columns of L = chol(C + sI), spread over a cluster.
// The k columns form 2*NC blocks of b columns ("players" of a round-robin
// tournament); CTA c plays the blocks at positions c (top slot) and 2NC-1-c
// (bottom slot), so every pair of blocks meets once per sweep of 2NC-1
// block-rounds. Block-round 0 of a sweep treats all pairs among the CTA's 2b
// columns (covering the pairs inside every block); later rounds only the b x b
// cross pairs, b disjoint pairs per inner round, one warp per pair. Between
// block-rounds the blocks move one position along the tournament circle: each
// CTA pushes its top block into the top slot of CTA c-1 and its bottom block
// into the bottom slot of CTA c+1 (distributed shared memory stores into the
// next of two slot buffers), then the cluster meets at one barrier. CTAs only
// synchronise through cluster barriers, taken the same number of times by all
// of them (no spin waits).
template <int NI, int EIG_THREADS>
__global__ void __launch_bounds__(EIG_THREADS, 1) k_eig_cluster(EigArgs a) {
  constexpr int EIG_WARPS = EIG_THREADS / 32;
  extern __shared__ __align__(16) float esm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int NC = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = a.k, b = a.b, kp = a.kp, nb = 2 * NC;
  const int slot = b * kp;  // floats per slot; buffer x starts at offset 2 * slot * x (top slot, then bottom)
  __shared__ int s_count, s_total;
  __shared__ unsigned s_off, s_offmax;  // largest squared pair cosine of a sweep (FP32 bits, >= 0)
  __shared__ unsigned s_absmax;         // largest |w_ij| of the CTA's blocks, then of the cluster (FP32 bits)
  if (tid == 0) { s_total = 0; s_offmax = 0u; s_absmax = 0u; }

  // ---- initial blocks (round 0 positions) from the factor ------------------
  // (asynchronous copies, all in flight at once; zero outside the factor)
  {
    const int blk[2] = {rr_player(rank, 0, nb), rr_player(nb - 1 - rank, 0, nb)};
    for (int sl = 0; sl < 2; ++sl) {
      const int c0 = min(k, blk[sl] * b), nc = min(k, c0 + b) - c0;
      const int dst = sl * slot;
      for (int e = tid; e < b * kp; e += EIG_THREADS) {
        const int c = e / kp, i = e % kp;
        const bool ok = c < nc && i < k && (a.full || i >= c0 + c);
        cp_async4(esm + dst + e, a.L + (ok ? (size_t)i * k + c0 + c : 0), ok);
      }
    }
    cp_async_wait_all();
  }
  // SVD input (a.full): exact power-of-two rescaling so that the largest entry
  // is in [0.5, 1), since products of squared column norms of a tiny-scale
  // matrix (the R factor of a factor scaled 1e-6, say) would otherwise
  // underflow in the pair tests. The eigensolver's Cholesky factor is used as
  // loaded (its validated path). a.full is uniform over the cluster, so every
  // CTA takes the same barriers.
  int wexp = 0;
  if (a.full) {
    __syncthreads();
    float m = 0.0f;
    for (int e = tid; e < 2 * slot; e += EIG_THREADS) m = fmaxf(m, fabsf(esm[e]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0 && m > 0.0f) atomicMax(&s_absmax, __float_as_uint(m));
    cluster.sync();  // every CTA's blocks are loaded and its maximum taken
    if (tid == 0 && s_absmax) atomicMax(cluster.map_shared_rank(&s_absmax, 0), s_absmax);
    cluster.sync();
    const float wmax = __uint_as_float(*cluster.map_shared_rank(&s_absmax, 0));
    frexpf(wmax, &wexp);  // wmax = f 2^wexp, f in [0.5, 1) (wexp = 0 for a zero matrix)
    const float wscale = ldexpf(1.0f, -wexp);
    for (int e = tid; e < 2 * slot; e += EIG_THREADS) esm[e] *= wscale;
  }
  // Every CTA has its blocks before the first distributed shared memory store.
  cluster.sync();

  // ---- sweeps ---------------------------------------------------------------
  // Squared column norms are cached next to the slots (recomputed at the start
  // of every sweep, updated by each rotation, moved with their columns).
  float* nrm = esm + 4 * slot;  // [buffer][slot][b]
  int sweep = 0, cur = 0, done = 0;
  for (; sweep < a.max_sweeps && !done; ++sweep) {
    if (tid == 0) { s_count = 0; s_off = 0u; }
    for (int c = warp; c < 2 * b; c += EIG_WARPS) {  // zero columns give zero norms
      float4 x[NI];
      col_load<NI>(esm, 2 * slot * cur + (c < b ? c * kp : slot + (c - b) * kp), x, lane);
      const float n2 = col_sumsq<NI>(x);
      if (lane == 0) nrm[(2 * cur + (c < b ? 0 : 1)) * b + (c < b ? c : c - b)] = n2;
    }
    __syncthreads();
    float off2 = 0.0f;
    for (int t = 0; t < nb - 1; ++t) {
      const int blkA = rr_player(rank, t, nb), blkB = rr_player(nb - 1 - rank, t, nb);
      const int ba = max(0, min(k, blkA * b + b) - blkA * b);
      const int bb = max(0, min(k, blkB * b + b) - blkB * b);
      const int top = 2 * slot * cur;
      const int bot = top + slot;
      float* ntop = nrm + 2 * cur * b;
      float* nbot = ntop + b;
      int cnt = 0;
      if (t == 0) {  // every pair among the ba + bb local columns
        const int n2 = ba + bb, m2 = n2 + (n2 & 1);
        for (int r = 0; r < m2 - 1; ++r) {
          for (int p = warp; p < m2 / 2; p += EIG_WARPS) {
            int u = rr_player(p, r, m2), v = rr_player(m2 - 1 - p, r, m2);
            if (u < n2 && v < n2) {
              const int cu = u < ba ? top + u * kp : bot + (u - ba) * kp;
              const int cv = v < ba ? top + v * kp : bot + (v - ba) * kp;
              float* nu = u < ba ? ntop + u : nbot + (u - ba);
              float* nv = v < ba ? ntop + v : nbot + (v - ba);
              float4 x[NI], y[NI];
              col_load<NI>(esm, cu, x, lane);
              col_load<NI>(esm, cv, y, lane);
              float al = *nu, be = *nv;
              if (jacobi_rot<NI>(x, y, al, be, a.tol, off2)) {
                col_store<NI>(esm, cu, x, lane);
                col_store<NI>(esm, cv, y, lane);
                if (lane == 0) { *nu = al; *nv = be; }
                ++cnt;
              }
            }
          }
          __syncthreads();
        }
      } else {  // the ba x bb cross pairs, max(ba, bb) disjoint pairs per inner round
        const int bmax = max(ba, bb);
        if (bmax <= EIG_WARPS) {
          // Warp i keeps top column i in registers for the whole block-round;
          // the bottom columns pass from warp to warp through shared memory.
          const int i = warp;
          const bool has_top = i < ba;
          float4 x[NI];
          float al = 0.0f;
          if (has_top) {
            col_load<NI>(esm, top + i * kp, x, lane);
            al = ntop[i];
          }
          for (int r = 0; r < bmax; ++r) {
            const int j = (i + r) % bmax;
            if (has_top && j < bb) {
              float4 y[NI];
              col_load<NI>(esm, bot + j * kp, y, lane);
              float be = nbot[j];
              if (jacobi_rot<NI>(x, y, al, be, a.tol, off2)) {
                col_store<NI>(esm, bot + j * kp, y, lane);
                if (lane == 0) nbot[j] = be;
                ++cnt;
              }
            }
            __syncthreads();
          }
          if (has_top) {
            col_store<NI>(esm, top + i * kp, x, lane);
            if (lane == 0) ntop[i] = al;
          }
          __syncthreads();
        } else {  // more pairs than warps: both columns through shared memory
          for (int r = 0; r < bmax; ++r) {
            for (int i = warp; i < bmax; i += EIG_WARPS) {
              const int j = (i + r) % bmax;
              if (i < ba && j < bb) {
                float4 x[NI], y[NI];
                col_load<NI>(esm, top + i * kp, x, lane);
                col_load<NI>(esm, bot + j * kp, y, lane);
                float al = ntop[i], be = nbot[j];
                if (jacobi_rot<NI>(x, y, al, be, a.tol, off2)) {
                  col_store<NI>(esm, top + i * kp, x, lane);
                  col_store<NI>(esm, bot + j * kp, y, lane);
                  if (lane == 0) { ntop[i] = al; nbot[j] = be; }
                  ++cnt;
                }
              }
            }
            __syncthreads();
          }
        }
      }
      if (lane == 0 && cnt) atomicAdd(&s_count, cnt);
      // Move the blocks one position along the circle (position 0 stays):
      // top of CTA c -> top of c-1 (CTA 1's top -> bottom of CTA 0), bottom of
      // CTA c -> bottom of c+1 (the last CTA's bottom -> its own top).
      if (NC > 1) {
        const int nxt = cur ^ 1;
        int dq_top, ds_top, dq_bot, ds_bot;  // destination CTA and slot
        if (rank == 0) { dq_top = 0; ds_top = 0; }
        else if (rank == 1) { dq_top = 0; ds_top = 1; }
        else { dq_top = rank - 1; ds_top = 0; }
        if (rank == NC - 1) { dq_bot = rank; ds_bot = 0; }
        else { dq_bot = rank + 1; ds_bot = 1; }
        float4* d1 = reinterpret_cast<float4*>(cluster.map_shared_rank(esm + 2 * slot * nxt + ds_top * slot, dq_top));
        float4* d2 = reinterpret_cast<float4*>(cluster.map_shared_rank(esm + 2 * slot * nxt + ds_bot * slot, dq_bot));
        const float4* s1 = reinterpret_cast<const float4*>(esm + top);
        const float4* s2 = reinterpret_cast<const float4*>(esm + bot);
        const int n4 = slot / 4;
        for (int e = tid; e < n4; e += EIG_THREADS) {
          d1[e] = s1[e];
          d2[e] = s2[e];
        }
        if (tid < b) {
          *cluster.map_shared_rank(nrm + (2 * nxt + ds_top) * b + tid, dq_top) = ntop[tid];
          *cluster.map_shared_rank(nrm + (2 * nxt + ds_bot) * b + tid, dq_bot) = nbot[tid];
        }
        cluster.sync();
        cur = nxt;
      }
    }
    if (lane == 0 && off2 > 0.0f) atomicMax(&s_off, __float_as_uint(off2));
    __syncthreads();  // every warp's count is in s_count (a 1-CTA cluster has no barrier above)
    // convergence: total rotations of the sweep over the cluster, and its
    // largest pair cosine (non-negative floats order as their bit patterns)
    if (tid == 0 && s_count) atomicAdd(cluster.map_shared_rank(&s_total, 0), s_count);
    if (tid == 0 && s_off) atomicMax(cluster.map_shared_rank(&s_offmax, 0), s_off);
    cluster.sync();
    const int total = *cluster.map_shared_rank(&s_total, 0);
    const float offmax = __uint_as_float(*cluster.map_shared_rank(&s_offmax, 0));
    cluster.sync();
    if (rank == 0 && tid == 0) { s_total = 0; s_offmax = 0u; }
    // Done when a sweep rotated nothing. Cyclic Jacobi converges quadratically:
    // a sweep that started with every pair cosine below stop_tol leaves them
    // near stop_tol^2, so the sweep that would only confirm it is skipped.
    done = total == 0 || (a.stop_tol > 0.0f && offmax <= a.stop_tol * a.stop_tol);
  }
  if (rank == 0 && tid == 0) {
    if (!done) raise_flag(a.flags, KFAC_FLAG_EIG_NOCONV);
    if (a.stats) {
      atomicAdd(a.stats + STAT_SWEEPS, (unsigned long long)sweep);
      atomicAdd(a.stats + STAT_EIG_SOLVES, 1ull);
    }
  }

  // ---- eigenpairs of the blocks held here: lam_j = |w_j|^2 - s, x_j = w_j / |w_j|
  // After a whole number of sweeps the blocks are back at their round-0 positions.
  const double sh = *a.shift;
  const double unscale = ldexp(1.0, 2 * wexp);  // |w_j|^2 back in the input's units
  const int blk[2] = {rr_player(rank, 0, nb), rr_player(nb - 1 - rank, 0, nb)};
  for (int sl = 0; sl < 2; ++sl) {
    const int c0 = blk[sl] * b;
    const float* base = esm + 2 * slot * cur + sl * slot;
    for (int c = warp; c < b; c += EIG_WARPS) {
      const int j = c0 + c;
      if (j >= k) continue;
      const float* wj = base + (size_t)c * kp;
      double n2 = 0.0;
      for (int i = lane; i < k; i += 32) n2 += (double)wj[i] * (double)wj[i];
      for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
      n2 = __shfl_sync(0xffffffffu, n2, 0);
      double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
      for (int i = lane; i < k; i += 32) a.X[(size_t)i * k + j] = (double)wj[i] * inv;
      if (lane == 0) a.lam[j] = n2 * unscale - sh;
    }
  }
  cluster.sync();  // no CTA leaves while others may still address its shared memory
}

// Refinement combine, spread over many CTAs (FP64 runs at ~2 operations per
// clock per SM, so one CTA would spend ~0.2 ms on the k^2 divisions):
//  k_refine_norms: lam_i = S_ii / (X^T X)_ii and per-CTA partial sums of
//    ||S - diag(lam)||_F^2, ||C||_F^2, ||R||_F^2 (R = I - X^T X);
//  k_refine_E: the separation threshold delta = 2 (||S - diag(lam)|| +
//    ||C|| ||R||) from the partials (same fixed order in every CTA), then
//    E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i) where |lam_j - lam_i| > delta,
//    R_ij / 2 otherwise.
constexpr int REF_THREADS = 256;
constexpr int REF_MAX_BLOCKS = 128;

__device__ __forceinline__ double block_sum_ref(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < REF_THREADS / 32; ++w) t += red[w];
  return t;  // valid in thread 0
}

__global__ void __launch_bounds__(REF_THREADS) k_refine_norms(const double* __restrict__ C,
                                                               const double* __restrict__ XtX,
                                                               const double* __restrict__ S, int k,
                                                               double* __restrict__ lam, double* __restrict__ part) {
  __shared__ double red[REF_THREADS / 32];
  const long long kk = (long long)k * k, step = (long long)gridDim.x * REF_THREADS;
  const long long g0 = (long long)blockIdx.x * REF_THREADS + threadIdx.x;
  if (g0 < k) lam[g0] = S[(size_t)g0 * k + g0] / XtX[(size_t)g0 * k + g0];  // S_ii / (1 - R_ii)
  double a = 0.0, b = 0.0, c = 0.0;
  for (long long e = g0; e < kk; e += step) {
    const int i = (int)(e / k), j = (int)(e - (long long)i * k);
    const double sv = S[e] - (i == j ? S[e] / XtX[e] : 0.0);
    const double rv = (i == j ? 1.0 : 0.0) - XtX[e];
    a = fma(sv, sv, a);
    b = fma(C[e], C[e], b);
    c = fma(rv, rv, c);
  }
  const double A = block_sum_ref(a, red);
  const double Bn = block_sum_ref(b, red);
  const double Cn = block_sum_ref(c, red);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x + 0] = A;
    part[3 * blockIdx.x + 1] = Bn;
    part[3 * blockIdx.x + 2] = Cn;
  }
}

__global__ void __launch_bounds__(REF_THREADS) k_refine_E(const double* __restrict__ XtX,
                                                           const double* __restrict__ S, int k,
                                                           const double* __restrict__ lam,
                                                           const double* __restrict__ part, int nparts,
                                                           double* __restrict__ E, int* flags) {
  __shared__ double s_delta;
  if (threadIdx.x < 32) {  // fixed order: lane-strided partials, then a fixed shuffle tree
    double A = 0.0, Bn = 0.0, Cn = 0.0;
    for (int p = threadIdx.x; p < nparts; p += 32) {
      A += part[3 * p];
      Bn += part[3 * p + 1];
      Cn += part[3 * p + 2];
    }
    for (int o = 16; o > 0; o >>= 1) {
      A += __shfl_xor_sync(0xffffffffu, A, o);
      Bn += __shfl_xor_sync(0xffffffffu, Bn, o);
      Cn += __shfl_xor_sync(0xffffffffu, Cn, o);
    }
    if (threadIdx.x == 0) {
      s_delta = 2.0 * (sqrt(A) + sqrt(Bn) * sqrt(Cn));
      if (blockIdx.x == 0 && !isfinite(s_delta)) raise_flag(flags, KFAC_FLAG_NONFINITE);
    }
  }
  __syncthreads();
  const double delta = s_delta;
  const long long kk = (long long)k * k, step = (long long)gridDim.x * REF_THREADS;
  for (long long e = (long long)blockIdx.x * REF_THREADS + threadIdx.x; e < kk; e += step) {
    const int i = (int)(e / k), j = (int)(e - (long long)i * k);
    const double rij = (i == j ? 1.0 : 0.0) - XtX[e];
    double v;
    if (i == j) {
      v = 0.5 * rij;
    } else {
      const double gap = lam[j] - lam[i];
      v = (fabs(gap) > delta) ? (S[e] + lam[j] * rij) / gap : 0.5 * rij;
    }
    E[e] = v;
  }
}

__global__ void __launch_bounds__(1024) k_eig_select(const double* __restrict__ X, const double* __restrict__ lam,
                                                      int k, int r, float lambda, float* __restrict__ Pt,
                                                      long long ldpt, float* __restrict__ D,
                                                      float* __restrict__ coef, float* __restrict__ Uout,
                                                      long long ldu, int singular) {
  // Every CTA ranks the k eigenvalues (from shared memory) and copies its
  // slice of the selected columns; CTA 0 also writes D and the coefficients.
  // Ranking compares order-preserving integer keys of the FP64 values (an
  // FP64 compare would run on the FP64 pipe at ~1/64 rate).
  extern __shared__ unsigned long long sel_sm[];
  unsigned long long* key = sel_sm;                 // k keys, NaN ranked last
  int* order = reinterpret_cast<int*>(sel_sm + k);  // order[rank] = index
  const int tid = threadIdx.x;
  for (int i = tid; i < k; i += blockDim.x) {
    const long long bits = __double_as_longlong(lam[i]);
    const bool nan = (bits & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
    key[i] = nan ? 0ull : (bits < 0 ? ~(unsigned long long)bits : (unsigned long long)bits | (1ull << 63));
  }
  __syncthreads();
  for (int i = tid; i < k; i += blockDim.x) {
    const unsigned long long ki = key[i];
    int rk = 0;
    for (int j = 0; j < k; ++j) {
      const unsigned long long kj = key[j];
      rk += (kj > ki) || (kj == ki && j < i);
    }
    order[rk] = i;
  }
  __syncthreads();
  if (blockIdx.x == 0) {
    for (int t = tid; t < r; t += blockDim.x) {
      double v = lam[order[t]];
      if (singular) v = sqrt(v > 0.0 ? v : 0.0);  // singular value from its square
      double dv = v > 0.0 ? v : 0.0;
      if (D) D[t] = (float)v;
      if (coef) coef[t] = (float)(1.0 / (dv + (double)lambda) - 1.0 / (double)lambda);
    }
  }
  const long long total = (long long)k * r, step = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + tid; e < total; e += step) {
    int row = (int)(e / r), t = (int)(e % r);
    float v = (float)X[(size_t)row * k + order[t]];
    if (Pt) Pt[(long long)t * ldpt + row] = v;
    if (Uout) Uout[(long long)row * ldu + t] = v;
  }
}

}  // namespace

template <int NI, int EIG_THREADS>
static cudaError_t launch_eig(const EigArgs& a, int nc, size_t smem, cudaStream_t s) {
  {
    cudaError_t e = set_kernel_attrs_once(reinterpret_cast<const void*>(k_eig_cluster<NI, EIG_THREADS>), kSmemOptin, true);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc, 1, 1);
  cfg.blockDim = dim3(EIG_THREADS, 1, 1);
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
  return cudaLaunchKernelEx(&cfg, k_eig_cluster<NI, EIG_THREADS>, a);
}

cudaError_t eig_jacobi_f32(const double* C, int k, double shift_rel, int max_sweeps, float tol, float stop_tol,
                           double* X, double* lam, float* gscratch, int* flags, unsigned long long* stats,
                           cudaStream_t s, const float* C32, long long ld32, int chol_nc, int chol_panel,
                           int chol_blocked_on, long long wait_cycles) {
  if (k <= 0) return cudaSuccess;
  // W = L with L L^T = C + sI, factorised in FP32; the shift it used (grown on
  // breakdown) is stored after the factor.
  double* shift = reinterpret_cast<double*>(gscratch + (((size_t)k * k + 1) & ~(size_t)1));
  cudaError_t e = (chol_blocked_on && C32 && chol_blocked_ws_bytes(k) > 0)
                      ? chol_blocked(C, C32, ld32, k, shift_rel, gscratch, flags, stats, s, shift,
                                     gscratch + eig_scratch_head_floats(k), wait_cycles)
                      : chol_cluster(C, k, shift_rel, /*fp64=*/false, gscratch, flags, stats, s, shift, C32, ld32,
                                     chol_nc, chol_panel);
  if (e != cudaSuccess) return e;
  return jacobi_columns(k, max_sweeps, tol, stop_tol, X, lam, gscratch, shift, flags, stats, s, 0);
}

cudaError_t svd_jacobi_f32(const float* W32, int k, int max_sweeps, float tol, float stop_tol, double* X, double* lam,
                           float* gscratch, int* flags, unsigned long long* stats, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  double* shift = reinterpret_cast<double*>(gscratch + (((size_t)k * k + 1) & ~(size_t)1));
  cudaError_t e = cudaMemcpyAsync(gscratch, W32, sizeof(float) * (size_t)k * k, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(shift, 0, sizeof(double), s)) != cudaSuccess) return e;
  return jacobi_columns(k, max_sweeps, tol, stop_tol, X, lam, gscratch, shift, flags, stats, s, 1);
}

cudaError_t jacobi_columns(int k, int max_sweeps, float tol, float stop_tol, double* X, double* lam, float* gscratch,
                           const double* shift, int* flags, unsigned long long* stats, cudaStream_t s, int full) {
  // b = ceil(k / 2nc) <= 8 where the cluster allows it: a cross round's b pairs
  // then leave each sub-partition at most two busy warps.
  int nc = (k + 15) / 16;
  nc = nc < 1 ? 1 : (nc > EIG_MAX_NC ? EIG_MAX_NC : nc);
  const int b = (k + 2 * nc - 1) / (2 * nc);
  const int kp = (k + 127) / 128 * 128;  // float4 per lane, 32 lanes
  const size_t smem = sizeof(float) * 4 * ((size_t)b * kp + b);  // 2 buffers x 2 slots, with their column norms
  if (smem > (size_t)kSmemOptin) return cudaErrorInvalidValue;
  EigArgs a = {gscratch, shift, k, max_sweeps, tol, X, lam, flags, stats, b, kp, stop_tol, full};
  if (b <= 8) {
    switch (kp / 128) {
      case 1: return launch_eig<1, 256>(a, nc, smem, s);
      case 2: return launch_eig<2, 256>(a, nc, smem, s);
      case 3: return launch_eig<3, 256>(a, nc, smem, s);
      case 4: return launch_eig<4, 256>(a, nc, smem, s);
      case 5: return launch_eig<5, 256>(a, nc, smem, s);
      default: return cudaErrorInvalidValue;
    }
  }
  // Blocks of 17 or 18 columns (k in (512, 576] on the 16-CTA limit): one warp
  // per pair needs 17-18 warps, so every column pair of an inner round runs at
  // once with the top column in registers (16 warps would take two passes with
  // both columns through shared memory).
  if (kp / 128 == 5 && b == 17) return launch_eig<5, 17 * 32>(a, nc, smem, s);
  if (kp / 128 == 5 && b == 18) return launch_eig<5, 18 * 32>(a, nc, smem, s);
  switch (kp / 128) {
    case 1: return launch_eig<1, EIG_THREADS_MAX>(a, nc, smem, s);
    case 2: return launch_eig<2, EIG_THREADS_MAX>(a, nc, smem, s);
    case 3: return launch_eig<3, EIG_THREADS_MAX>(a, nc, smem, s);
    case 4: return launch_eig<4, EIG_THREADS_MAX>(a, nc, smem, s);
    case 5: return launch_eig<5, EIG_THREADS_MAX>(a, nc, smem, s);
    default: return cudaErrorInvalidValue;
  }
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
  {
    const long long kk2 = (long long)k * k;
    int nb = (int)((kk2 + 4 * REF_THREADS - 1) / (4 * REF_THREADS));
    nb = nb < 1 ? 1 : (nb > REF_MAX_BLOCKS ? REF_MAX_BLOCKS : nb);
    double* part = work + 5 * kk;  // 3 * REF_MAX_BLOCKS doubles after the five k x k blocks
    k_refine_norms<<<nb, REF_THREADS, 0, s>>>(C, XtX, S, k, lam, part);
    note_launch();
    k_refine_E<<<nb, REF_THREADS, 0, s>>>(XtX, S, k, lam, part, nb, E, flags);
  }
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // Xn = X + X E
  g.A = X; g.sam = k; g.sak = 1; g.B = E; g.sbn = 1; g.sbk = k; g.D = Xn; g.ldd = k; g.beta = 1.0; g.C0 = X;
  g.ldc = k;
  if ((e = gemm_simt_f64(g, s)) != cudaSuccess) return e;
  return cudaMemcpyAsync(X, Xn, kk * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

namespace {
__global__ void k_polish_factor(double* __restrict__ G, int k) {
  const long long kk = (long long)k * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < kk; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), j = (int)(e - (long long)i * k);
    G[e] = (i == j ? 1.5 : 0.0) - 0.5 * G[e];
  }
}
__global__ void k_f64_to_f32(const double* __restrict__ in, long long n, float* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = (float)in[e];
}

// ---- FP32 refinement and polish (k x k) ------------------------------------
// The FP32 work matrices have the row stride ld = ref_ld(k) (a multiple of 4
// floats), so their products qualify for the tensor cores.
// X (FP64, row stride k) -> X32 = X and Xt32 = X^T in FP32, 32 x 32 tiles
// through shared memory (both stores coalesced).
__global__ void k_split_f32_t(const double* __restrict__ X, int k, float* __restrict__ X32, float* __restrict__ Xt32,
                              long long ld) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32, tx = threadIdx.x;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = r0 + y, c = c0 + tx;
    float v = 0.0f;
    if (r < k && c < k) {
      v = (float)X[(size_t)r * k + c];
      if (X32) X32[(size_t)r * ld + c] = v;
    }
    tile[y][tx] = v;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y, r = r0 + tx;  // Xt32[c][r] = X[r][c]
    if (r < k && c < k) Xt32[(size_t)c * ld + r] = tile[tx][y];
  }
}

// dst (k x k, row stride ldd) = src (row stride lds).
__global__ void k_copy_f32(const float* __restrict__ src, long long lds, int k, float* __restrict__ dst, long long ldd) {
  const long long n = (long long)k * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), j = (int)(e - (long long)i * k);
    dst[(size_t)i * ldd + j] = src[(size_t)i * lds + j];
  }
}

// lam_i = S_ii / G_ii (G = X^T X) and per-CTA partial sums of ||S - diag(lam)||^2,
// ||C||^2, ||I - G||^2; a CTA takes whole rows.
__global__ void __launch_bounds__(REF_THREADS) k_refine_norms32(const float* __restrict__ C32, long long ldc32,
                                                                 const float* __restrict__ G,
                                                                 const float* __restrict__ S, int k, long long ld,
                                                                 double* __restrict__ lam, double* __restrict__ part) {
  __shared__ double red[REF_THREADS / 32];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = blockIdx.x; i < k; i += gridDim.x) {
    const float* Si = S + (size_t)i * ld;
    const float* Gi = G + (size_t)i * ld;
    const float* Ci = C32 + (size_t)i * ldc32;
    if (threadIdx.x == 0) lam[i] = (double)Si[i] / (double)Gi[i];
    for (int j = threadIdx.x; j < k; j += REF_THREADS) {
      const double sv = i == j ? (double)Si[i] - (double)Si[i] / (double)Gi[i] : (double)Si[j];  // S - diag(lam)
      const float rv = (i == j ? 1.0f : 0.0f) - Gi[j];
      a = fma(sv, sv, a);
      b = fma((double)Ci[j], (double)Ci[j], b);
      c = fma((double)rv, (double)rv, c);
    }
  }
  const double A = block_sum_ref(a, red);
  const double Bn = block_sum_ref(b, red);
  const double Cn = block_sum_ref(c, red);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x + 0] = A;
    part[3 * blockIdx.x + 1] = Bn;
    part[3 * blockIdx.x + 2] = Cn;
  }
}

// E^T (FP32): E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i) for separated
// pairs, R_ij / 2 otherwise (R = I - G); the threshold as k_refine_E.
__global__ void __launch_bounds__(REF_THREADS) k_refine_Et32(const float* __restrict__ G, const float* __restrict__ S,
                                                              int k, long long ld, const double* __restrict__ lam,
                                                              const double* __restrict__ part, int nparts,
                                                              float* __restrict__ Et, int* flags) {
  __shared__ double s_delta;
  if (threadIdx.x < 32) {
    double A = 0.0, Bn = 0.0, Cn = 0.0;
    for (int p = threadIdx.x; p < nparts; p += 32) {
      A += part[3 * p];
      Bn += part[3 * p + 1];
      Cn += part[3 * p + 2];
    }
    for (int o = 16; o > 0; o >>= 1) {
      A += __shfl_xor_sync(0xffffffffu, A, o);
      Bn += __shfl_xor_sync(0xffffffffu, Bn, o);
      Cn += __shfl_xor_sync(0xffffffffu, Cn, o);
    }
    if (threadIdx.x == 0) {
      s_delta = 2.0 * (sqrt(A) + sqrt(Bn) * sqrt(Cn));
      if (blockIdx.x == 0 && !isfinite(s_delta)) raise_flag(flags, KFAC_FLAG_NONFINITE);
    }
  }
  __syncthreads();
  const float delta = (float)s_delta;
  for (int j = blockIdx.x; j < k; j += gridDim.x) {  // row j of E^T = column j of E
    const float lj = (float)lam[j];
    for (int i = threadIdx.x; i < k; i += REF_THREADS) {
      const float rij = (i == j ? 1.0f : 0.0f) - G[(size_t)i * ld + j];
      float v;
      if (i == j) {
        v = 0.5f * rij;
      } else {
        const float gap = (float)(lam[j] - lam[i]);
        v = (fabsf(gap) > delta) ? __fdiv_rn(fmaf(lj, rij, S[(size_t)i * ld + j]), gap) : 0.5f * rij;
      }
      Et[(size_t)j * ld + i] = v;
    }
  }
}

// X += alpha * D (FP64 X with row stride k, FP32 D with row stride ld), k x k.
__global__ void k_axpy_f64_f32(double* __restrict__ X, const float* __restrict__ D, int k, long long ld, double alpha) {
  const long long n = (long long)k * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), j = (int)(e - (long long)i * k);
    X[e] = fma(alpha, (double)D[(size_t)i * ld + j], X[e]);
  }
}

// E32 = G - I in FP32 (from the FP64 Gram, so the diagonal keeps its small part).
__global__ void k_polish_E32(const double* __restrict__ G, int k, float* __restrict__ E32, long long ld) {
  for (int i = blockIdx.x; i < k; i += gridDim.x)
    for (int j = threadIdx.x; j < k; j += blockDim.x)
      E32[(size_t)i * ld + j] = (float)(G[(size_t)i * k + j] - (i == j ? 1.0 : 0.0));
}

// C <- C - (P + P^T)/2 + (Q + Q^T)/8 with P = E C and Q = E C E: the same
// symmetric result as M C M for M = I - E/2, and C32 = C (row stride k).
__global__ void k_polish_apply(double* __restrict__ C, const float* __restrict__ P, const float* __restrict__ Q,
                               int k, long long ld, float* __restrict__ C32) {
  for (int i = blockIdx.x; i < k; i += gridDim.x)
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
      const size_t ij = (size_t)i * ld + j, ji = (size_t)j * ld + i;
      const double v = C[(size_t)i * k + j] - 0.5 * ((double)P[ij] + (double)P[ji]) +
                       0.125 * ((double)Q[ij] + (double)Q[ji]);
      C[(size_t)i * k + j] = v;
      C32[(size_t)i * k + j] = (float)v;
    }
}
}  // namespace

cudaError_t polish_factor(double* G, int k, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  const long long kk = (long long)k * k;
  const int grid = (int)std::min<long long>(304, (kk + 255) / 256);
  k_polish_factor<<<grid, 256, 0, s>>>(G, k);
  note_launch();
  return cudaGetLastError();
}

cudaError_t convert_f64_to_f32(const double* in, long long n, float* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::min<long long>(304, (n + 255) / 256);
  k_f64_to_f32<<<grid, 256, 0, s>>>(in, n, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t eig_select(const double* X, const double* lam, int k, int r, float lambda, float* Pt, long long ldpt,
                       float* D, float* coef, float* Uout, long long ldu, cudaStream_t s, int singular) {
  if (k <= 0) return cudaSuccess;
  const long long total = (long long)k * r;
  int grid = (int)((total + 4095) / 4096);
  grid = grid < 1 ? 1 : (grid > 152 ? 152 : grid);
  k_eig_select<<<grid, 1024, (sizeof(double) + sizeof(int)) * k + 8, s>>>(X, lam, k, r, lambda, Pt, ldpt, D, coef,
                                                                           Uout, ldu, singular);
  note_launch();
  return cudaGetLastError();
}


namespace {
// D (k x k) = A B^T for row-major FP32 A and B, all with row stride ld: FP32-
// accurate tensor-core products (3xTF32) from k = 128 up, the SIMT kernel below.
cudaError_t small_nt(const float* A, const float* B, float* D, int k, long long ld, bool d_trans, int* flags,
                     cudaStream_t s) {
  GemmDesc<float> g = {};
  g.M = k; g.N = k; g.K = k; g.alpha = 1.0f; g.beta = 0.0f; g.zsplit = 1;
  g.A = A; g.sam = ld; g.sak = 1;
  g.B = B; g.sbn = ld; g.sbk = 1;
  g.D = D; g.ldd = ld; g.d_trans = d_trans ? 1 : 0;
  g.flags = flags;
  if (k >= 128) return gemm_f32(g, KFAC_PREC_FP32, s);
  return gemm_small_f32(g, s);
}
int row_grid(int k) { return k < 1 ? 1 : (k > REF_MAX_BLOCKS ? REF_MAX_BLOCKS : k); }
int elem_grid(long long n) { return (int)std::min<long long>(304, std::max<long long>(1, (n + 255) / 256)); }
}  // namespace

cudaError_t eig_refine_f32(const float* C32, long long ldc32, int k, double* X, double* lam, float* w32, double* part,
                           int* flags, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  const long long ld = ref_ld(k);
  const size_t kl = (size_t)k * ld;
  float* X32 = w32;
  float* Xt = w32 + kl;
  float* G = w32 + 2 * kl;
  float* CXt = w32 + 3 * kl;
  float* S = w32 + 4 * kl;
  float* Et = w32 + 5 * kl;
  float* XE = w32 + 6 * kl;
  float* Cp = w32 + 7 * kl;  // C32 with the padded row stride
  const dim3 tg((k + 31) / 32, (k + 31) / 32);
  k_split_f32_t<<<tg, dim3(32, 8), 0, s>>>(X, k, X32, Xt, ld);
  note_launch();
  k_copy_f32<<<elem_grid((long long)k * k), 256, 0, s>>>(C32, ldc32, k, Cp, ld);
  note_launch();
  cudaError_t e;
  if ((e = small_nt(Xt, Xt, G, k, ld, false, flags, s)) != cudaSuccess) return e;   // G = X^T X
  if ((e = small_nt(Cp, Xt, CXt, k, ld, true, flags, s)) != cudaSuccess) return e;  // (C X)^T
  if ((e = small_nt(Xt, CXt, S, k, ld, false, flags, s)) != cudaSuccess) return e;  // S = X^T C X
  const int nb = row_grid(k);
  k_refine_norms32<<<nb, REF_THREADS, 0, s>>>(Cp, ld, G, S, k, ld, lam, part);
  note_launch();
  k_refine_Et32<<<nb, REF_THREADS, 0, s>>>(G, S, k, ld, lam, part, nb, Et, flags);
  note_launch();
  if ((e = small_nt(X32, Et, XE, k, ld, false, flags, s)) != cudaSuccess) return e;  // X E
  k_axpy_f64_f32<<<elem_grid((long long)k * k), 256, 0, s>>>(X, XE, k, ld, 1.0);
  note_launch();
  return cudaGetLastError();
}

cudaError_t polish_projected_f32(const double* G, double* C, float* C32, int k, float* w32, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  const long long ld = ref_ld(k);
  const size_t kl = (size_t)k * ld;
  float* E = w32;  // kept for polish_vectors_f32
  float* P = w32 + kl;
  float* Q = w32 + 2 * kl;
  float* Cp = w32 + 3 * kl;
  const int nb = row_grid(k);
  k_polish_E32<<<nb, 256, 0, s>>>(G, k, E, ld);
  note_launch();
  k_copy_f32<<<elem_grid((long long)k * k), 256, 0, s>>>(C32, k, k, Cp, ld);
  note_launch();
  cudaError_t e;
  if ((e = small_nt(E, Cp, P, k, ld, false, nullptr, s)) != cudaSuccess) return e;  // P = E C (C symmetric)
  if ((e = small_nt(P, E, Q, k, ld, false, nullptr, s)) != cudaSuccess) return e;   // Q = P E (E symmetric)
  k_polish_apply<<<nb, 256, 0, s>>>(C, P, Q, k, ld, C32);
  note_launch();
  return cudaGetLastError();
}

cudaError_t polish_E_f32(const double* G, int k, float* w32, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_polish_E32<<<row_grid(k), 256, 0, s>>>(G, k, w32, ref_ld(k));
  note_launch();
  return cudaGetLastError();
}

cudaError_t polish_vectors_f32(double* X, int k, float* w32, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  const long long ld = ref_ld(k);
  const size_t kl = (size_t)k * ld;
  const float* E = w32;
  float* Xt = w32 + kl;
  float* EX = w32 + 2 * kl;
  const dim3 tg((k + 31) / 32, (k + 31) / 32);
  k_split_f32_t<<<tg, dim3(32, 8), 0, s>>>(X, k, nullptr, Xt, ld);
  note_launch();
  cudaError_t e;
  if ((e = small_nt(E, Xt, EX, k, ld, false, nullptr, s)) != cudaSuccess) return e;  // E X
  k_axpy_f64_f32<<<elem_grid((long long)k * k), 256, 0, s>>>(X, EX, k, ld, -0.5);
  note_launch();
  return cudaGetLastError();
}

}  // namespace kfac
