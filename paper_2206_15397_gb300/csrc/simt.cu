// SIMT kernels: strided GEMM (FP32 with optional operand rounding, FP64),
// split-K reduction to FP64, transpose and widening copies.
#include <algorithm>
#include <mutex>
#include <set>
#include <utility>

#include "common.cuh"

namespace kfac {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// 64x64 output tile per CTA, 16x16 threads, each thread owns a 4x4 grid of
// outputs strided by 16 so that stores of consecutive threads are consecutive.
template <typename T, Round R>
__global__ void __launch_bounds__(NT) k_gemm_simt(GemmDesc<T> g) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int bm = blockIdx.y * BM, bn = blockIdx.x * BN;
  if (g.sym && bm > bn + BN - 1) return;  // tile strictly below the diagonal
  const int kbeg = blockIdx.z * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int it = 0; it < (BM * BK) / NT; ++it) {
      int e = tid + it * NT, mm, kk;
      if (g.sak == 1) { mm = e / BK; kk = e % BK; } else { mm = e % BM; kk = e / BM; }
      int m = bm + mm, k = k0 + kk;
      T v = T(0);
      if (m < g.M && k < kend) v = g.A[(long long)m * g.sam + (long long)k * g.sak];
      if constexpr (sizeof(T) == 4) v = round_operand(v, R);
      As[kk][mm] = v;
    }
#pragma unroll
    for (int it = 0; it < (BN * BK) / NT; ++it) {
      int e = tid + it * NT, nn, kk;
      if (g.sbk == 1) { nn = e / BK; kk = e % BK; } else { nn = e % BN; kk = e / BN; }
      int n = bn + nn, k = k0 + kk;
      T v = T(0);
      if (n < g.N && k < kend) v = g.B[(long long)n * g.sbn + (long long)k * g.sbk];
      if constexpr (sizeof(T) == 4) v = round_operand(v, R);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int m = bm + ty + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = bn + tx + 16 * j;
      if (n >= g.N) continue;
      if (g.sym && m > n) continue;
      T v = acc[i][j];
      if (g.zsplit <= 1) {
        v *= g.alpha;
        if (g.rowscale) v *= g.rowscale[m];
        if (g.colscale) v *= g.colscale[n];
        if (g.beta != T(0))
          v = fma(g.beta, g.C0[g.c0_trans ? (long long)n * g.ldc + m : (long long)m * g.ldc + n], v);
      }
      T* D = g.D + (g.zsplit > 1 ? blockIdx.z * g.zstride : 0);
      D[g.d_trans ? (long long)n * g.ldd + m : (long long)m * g.ldd + n] = v;
      if (g.sym && m != n) D[g.d_trans ? (long long)m * g.ldd + n : (long long)n * g.ldd + m] = v;
    }
  }
}

template <typename T, Round R>
cudaError_t launch_gemm(const GemmDesc<T>& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  GemmDesc<T> d = g;
  if (d.zsplit < 1) d.zsplit = 1;
  if (d.zsplit == 1) d.kchunk = d.K > 0 ? d.K : 1;
  dim3 grid((d.N + BN - 1) / BN, (d.M + BM - 1) / BM, d.zsplit);
  k_gemm_simt<T, R><<<grid, NT, 0, s>>>(d);
  note_launch();
  return cudaGetLastError();
}

// Small GEMM with 16 x 16 output tiles, one output per thread, for k x k
// products (k = 230 gives 225 CTAs): FP64 issues at ~2 FMA/clock/SM on this
// part, and a k x k FP32 product is latency-bound, so small tiles spread it
// over as many SMs as possible.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_t16(GemmDesc<T> g) {
  __shared__ T As[16][17];
  __shared__ T Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m = blockIdx.y * 16 + ty, n = blockIdx.x * 16 + tx;
  T acc = T(0);
  for (int k0 = 0; k0 < g.K; k0 += 16) {
    {  // A tile: element (row ty, k tx) or transposed pattern for coalescing
      int mm = ty, kk = tx;
      if (g.sak != 1) { mm = tx; kk = ty; }
      int am = blockIdx.y * 16 + mm, ak = k0 + kk;
      As[mm][kk] = (am < g.M && ak < g.K) ? g.A[(long long)am * g.sam + (long long)ak * g.sak] : T(0);
      int nn = ty, kb = tx;
      if (g.sbk != 1) { nn = tx; kb = ty; }
      int bn = blockIdx.x * 16 + nn, bk = k0 + kb;
      Bs[nn][kb] = (bn < g.N && bk < g.K) ? g.B[(long long)bn * g.sbn + (long long)bk * g.sbk] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc = fma(As[ty][kk], Bs[tx][kk], acc);
    __syncthreads();
  }
  if (m < g.M && n < g.N) {
    T v = acc * g.alpha;
    if (g.rowscale) v *= g.rowscale[m];
    if (g.colscale) v *= g.colscale[n];
    if (g.beta != T(0)) v = fma(g.beta, g.C0[g.c0_trans ? (long long)n * g.ldc + m : (long long)m * g.ldc + n], v);
    g.D[g.d_trans ? (long long)n * g.ldd + m : (long long)m * g.ldd + n] = v;
  }
}

// Sum of the split-K partials of entry (i, j) with Neumaier's compensated
// summation in FP32 (the FP64 pipe issues at ~1/64 of the FP32 rate on this
// part): s + c carries the sum to about FP64 accuracy for same-sign terms and
// to ~2u |sum| + nu^2 sum|x| in general.
// Loads go out eight at a time (each waits out the L2 latency otherwise).
__device__ __forceinline__ double sum_partials(const float* __restrict__ p, int nsplit, long long zstride) {
  float s = 0.0f, c = 0.0f;
  for (int z0 = 0; z0 < nsplit; z0 += 8) {
    float x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = z0 + q < nsplit ? p[(z0 + q) * zstride] : 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float t = s + x[q];
      c += (fabsf(s) >= fabsf(x[q])) ? (s - t) + x[q] : (x[q] - t) + s;
      s = t;
    }
  }
  return (double)s + (double)c;
}

// FP32 16 x 16-tile product for K <= kT16MaxK: both K-panels are staged in
// shared memory with all loads in flight at once, then one barrier (the
// per-16-column stepping of k_gemm_t16 waits out the global latency ~K/16 times).
constexpr int kT16MaxK = 256;
__global__ void __launch_bounds__(256) k_gemm_t16_wholek(GemmDesc<float> g) {
  __shared__ float As[16][kT16MaxK + 1];
  __shared__ float Bs[16][kT16MaxK + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int mb = blockIdx.y * 16, nb = blockIdx.x * 16;
  const int tot = 16 * g.K;
  for (int e0 = 0; e0 < tot; e0 += 8 * 256) {  // eight loads of each operand in flight per thread
    float va[8], vb[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = e0 + q * 256 + tid;
      va[q] = vb[q] = 0.0f;
      if (e < tot) {
        int r, kk;
        if (g.sak == 1) { r = e / g.K; kk = e - r * g.K; } else { kk = e >> 4; r = e & 15; }  // coalesced either way
        if (mb + r < g.M) va[q] = g.A[(long long)(mb + r) * g.sam + (long long)kk * g.sak];
        int rb, kb;
        if (g.sbk == 1) { rb = e / g.K; kb = e - rb * g.K; } else { kb = e >> 4; rb = e & 15; }
        if (nb + rb < g.N) vb[q] = g.B[(long long)(nb + rb) * g.sbn + (long long)kb * g.sbk];
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = e0 + q * 256 + tid;
      if (e < tot) {
        int r, kk;
        if (g.sak == 1) { r = e / g.K; kk = e - r * g.K; } else { kk = e >> 4; r = e & 15; }
        As[r][kk] = va[q];
        int rb, kb;
        if (g.sbk == 1) { rb = e / g.K; kb = e - rb * g.K; } else { kb = e >> 4; rb = e & 15; }
        Bs[rb][kb] = vb[q];
      }
    }
  }
  __syncthreads();
  const int m = mb + ty, n = nb + tx;
  float acc = 0.0f;
#pragma unroll 8
  for (int kk = 0; kk < g.K; ++kk) acc = fmaf(As[ty][kk], Bs[tx][kk], acc);
  if (m < g.M && n < g.N) {
    float v = acc * g.alpha;
    if (g.rowscale) v *= g.rowscale[m];
    if (g.colscale) v *= g.colscale[n];
    if (g.beta != 0.0f) v = fmaf(g.beta, g.C0[g.c0_trans ? (long long)n * g.ldc + m : (long long)m * g.ldc + n], v);
    g.D[g.d_trans ? (long long)n * g.ldd + m : (long long)m * g.ldd + n] = v;
  }
}

__device__ __forceinline__ double column_scale(double g) { return (isfinite(g) && g > 0.0) ? sqrt(g) : 1.0; }

// dscale[i] = sqrt(S_ii) of the summed partials (1 where S_ii is not positive
// and finite), summed in the same order as the reduce below sums S_ii
__global__ void k_diag_scale(const float* __restrict__ part, int nsplit, long long zstride, int n, int ldp,
                             double* __restrict__ dscale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dscale[i] = column_scale(sum_partials(part + (long long)i * ldp + i, nsplit, zstride));
}

__global__ void k_reduce_splitk(const float* __restrict__ part, int nsplit, long long zstride, int n, int ldp,
                                double* __restrict__ out, int ldo, int symmetrize, float* __restrict__ out32,
                                int* flags, const double* __restrict__ dscale) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // n * n < 2^31
  if (idx >= n * n) return;
  const int i = idx / n, j = idx - i * n;
  // symmetrize == 2: the partials hold the upper triangle only (a symmetric
  // product computed on the tiles at and above the diagonal); both halves of
  // the result read it, so the sum is exactly symmetric.
  const int a = symmetrize == 2 ? min(i, j) : i, b = symmetrize == 2 ? max(i, j) : j;
  double s = sum_partials(part + (long long)a * ldp + b, nsplit, zstride);
  if (!isfinite(s)) raise_flag(flags, KFAC_FLAG_NONFINITE);
  if (dscale) s /= dscale[i] * dscale[j];  // column scaling (k_diag_scale ran first)
  out[(long long)i * ldo + j] = s;
  if (out32 && symmetrize != 1) out32[(long long)i * n + j] = (float)s;  // FP32 copy for FP32 consumers (n x n, dense)
}

// out <- (out + out^T) / 2 in place, one thread per pair i <= j (the summed
// matrix is read twice, not the split-K partials), with the FP32 copy.
__global__ void k_symmetrize(double* __restrict__ out, int n, int ldo, float* __restrict__ out32) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int i = idx / n, j = idx - i * n;
  if (j < i) return;
  const double v = 0.5 * (out[(long long)i * ldo + j] + out[(long long)j * ldo + i]);
  out[(long long)i * ldo + j] = v;
  out[(long long)j * ldo + i] = v;
  if (out32) {
    out32[(long long)i * n + j] = (float)v;
    out32[(long long)j * n + i] = (float)v;
  }
}

// out[c][r] = in[r][c], or in[r][c] / rdiv[r] when rdiv is given
__global__ void k_transpose(const float* __restrict__ in, long long ldi, int rows, int cols, float* __restrict__ out,
                            long long ldo, const double* __restrict__ rdiv) {
  __shared__ float tile[32][33];
  int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    int r = r0 + y, c = c0 + threadIdx.x;
    if (r < rows && c < cols) {
      const float v = in[(long long)r * ldi + c];
      tile[y][threadIdx.x] = rdiv ? (float)((double)v / rdiv[r]) : v;
    }
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    int c = c0 + y, r = r0 + threadIdx.x;  // out[c][r] = in[r][c]
    if (r < rows && c < cols) out[(long long)c * ldo + r] = tile[threadIdx.x][y];
  }
}

// dst (rows x ldd, ldd a multiple of 4, 16-byte aligned) <- src (rows x cols,
// any row stride); columns cols..ldd-1 are zeroed. Each thread writes one
// 16-byte group, so the stores are vector stores whatever the source stride.
__global__ void k_pack_rows(const float* __restrict__ src, long long lds, int rows, int cols,
                            float* __restrict__ dst, long long ldd) {
  const long long groups = ldd >> 2, total = (long long)rows * groups;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long r = g / groups;
    const int c = (int)(g - r * groups) * 4;
    const float* s = src + r * lds;
    float4 v;
    v.x = c < cols ? s[c] : 0.0f;
    v.y = c + 1 < cols ? s[c + 1] : 0.0f;
    v.z = c + 2 < cols ? s[c + 2] : 0.0f;
    v.w = c + 3 < cols ? s[c + 3] : 0.0f;
    *reinterpret_cast<float4*>(dst + r * ldd + c) = v;
  }
}

// X (d x ldx, d = cols + append_one) <- scale * A^T for a row-major batch A
// (n x cols, row stride lda), with a last row of ones when append_one; the pad
// columns n..ldx-1 are zeroed. 32 x 32 tiles through shared memory so that both
// the reads of A and the writes of X are coalesced.
__global__ void k_rows_to_cols(const float* __restrict__ A, long long lda, int n, int cols, int append_one,
                               float scale, float* __restrict__ X, long long ldx) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.y * 32, t0 = blockIdx.x * 32;  // feature (row of X) and sample (column of X) blocks
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int t = t0 + y, c = c0 + threadIdx.x;
    tile[y][threadIdx.x] = (t < n && c < cols) ? scale * A[(long long)t * lda + c] : 0.0f;
  }
  __syncthreads();
  const int d = cols + append_one;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y, t = t0 + threadIdx.x;  // X[c][t] = A[t][c]
    if (c < d && t < ldx) X[(long long)c * ldx + t] = (t >= n) ? 0.0f : (c < cols ? tile[threadIdx.x][y] : 1.0f);
  }
}

// Patch matrix of a convolution input for samples [i0, i0 + ns): row
// (ch * kh + r) * kw + t, column (i - i0) * ho * wo + oy * wo + ox holds
// scale * x[i, ch, oy * sh + r - ph, ox * sw + t - pw] (0 outside the image);
// with append_one a last row of `scale`; columns past ns * ho * wo zeroed. One
// thread per column and row: consecutive threads take consecutive output
// positions, so the writes are coalesced and the reads strided by sw.
__global__ void k_im2col(const float* __restrict__ x, int c, int h, int w, int kh, int kw, int sh, int sw, int ph,
                         int pw, int ho, int wo, int i0, int ns, int append_one, float scale, float* __restrict__ X,
                         long long ldx) {
  const long long col = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int row = blockIdx.y;
  if (col >= ldx) return;
  const long long pos = (long long)ho * wo, ncols = (long long)ns * pos;
  float v = 0.0f;
  if (col < ncols) {
    if (append_one && row == c * kh * kw) {
      v = scale;
    } else {
      const int i = i0 + (int)(col / pos);
      const int q = (int)(col % pos), oy = q / wo, ox = q % wo;
      const int ch = row / (kh * kw), rt = row % (kh * kw), r = rt / kw, t = rt % kw;
      const int y = oy * sh + r - ph, xx = ox * sw + t - pw;
      if (y >= 0 && y < h && xx >= 0 && xx < w) v = scale * x[(((long long)i * c + ch) * h + y) * w + xx];
    }
  }
  X[(long long)row * ldx + col] = v;
}

// BF16 copy with a padded row stride: one thread per 8 outputs (a 16-byte store).
__global__ void k_to_bf16(const float* __restrict__ src, long long lds, int rows, int cols,
                          uint4* __restrict__ dst, long long ldd8) {
  const long long total = (long long)rows * ldd8;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long r = g / ldd8;
    const int c = (int)(g - r * ldd8) * 8;
    const float* sr = src + r * lds;
    unsigned u[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float a = c + 2 * q < cols ? sr[c + 2 * q] : 0.0f, b = c + 2 * q + 1 < cols ? sr[c + 2 * q + 1] : 0.0f;
      asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(u[q]) : "f"(b), "f"(a));
    }
    dst[g] = make_uint4(u[0], u[1], u[2], u[3]);
  }
}

__global__ void k_convert(const float* __restrict__ in, long long ldi, int rows, int cols, double* __restrict__ out,
                          long long ldo, int* flags) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)rows * cols) return;
  int r = (int)(idx / cols), c = (int)(idx % cols);
  float v = in[(long long)r * ldi + c];
  if (!isfinite(v)) raise_flag(flags, KFAC_FLAG_NONFINITE);
  out[(long long)r * ldo + c] = (double)v;
}

// Philox4x32 with 10 rounds (Salmon, Moraes, Dror and Shaw, SC'11): each round
// forms the two 32x32 -> 64-bit products of words 0 and 2 with the round
// multipliers, crosses their high halves with words 1 and 3 and the key, and
// steps the key by the Weyl increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Value e of the test-matrix stream: block e / 4 of Philox (counter (block, 0, 1)),
// two Box-Muller pairs per block, each word mapped to (floor(w / 512) + 1/2) / 2^23.
__device__ __forceinline__ float omega_value(unsigned long long e, uint32_t k0, uint32_t k1) {
  const unsigned long long b = e >> 2;
  const uint4 w = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)(b >> 32), 0u, 1u), k0, k1);
  const int t = (int)(e & 3);
  const uint32_t wu = t < 2 ? w.x : w.z, wv = t < 2 ? w.y : w.w;
  const float u = ((float)(wu >> 9) + 0.5f) * 0x1p-23f;  // exact in FP32: a 23-bit integer + 1/2, times 2^-23
  const float v = ((float)(wv >> 9) + 0.5f) * 0x1p-23f;
  const float rho = sqrtf(-2.0f * logf(u));
  float sn, cs;
  sincospif(2.0f * v, &sn, &cs);
  return rho * ((t & 1) ? sn : cs);
}

// Columns j0 .. j0 + ncols - 1 of the d x k seeded test matrix: out[i][j - j0], or
// with trans out[j - j0][i] (consecutive threads take consecutive i, so the
// transposed rows are written contiguously).
__global__ void k_draw_omega(int d, int k, int j0, int ncols, uint32_t k0, uint32_t k1, float* __restrict__ out,
                             long long ld, int trans) {
  const long long n = (long long)d * ncols;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
    long long i, j;
    if (trans) { j = x / d; i = x - j * d; }
    else { i = x / ncols; j = x - i * ncols; }
    const float z = omega_value((unsigned long long)i * (unsigned long long)k + (unsigned long long)(j0 + j), k0, k1);
    if (trans) out[j * ld + i] = z;
    else out[i * ld + j] = z;
  }
}

}  // namespace

cudaError_t draw_omega_f32(int d, int k, unsigned long long seed, int j0, int ncols, float* out, long long ld,
                           bool trans, cudaStream_t s) {
  if (d <= 0 || ncols <= 0) return cudaSuccess;
  const long long total = (long long)d * ncols;
  const long long blocks = std::min<long long>((total + 255) / 256, 152LL * 16);
  k_draw_omega<<<(unsigned)blocks, 256, 0, s>>>(d, k, j0, ncols, (uint32_t)seed, (uint32_t)(seed >> 32), out, ld,
                                                trans ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

cudaError_t set_kernel_attrs_once(const void* fn, int max_dyn_smem, bool nonportable_cluster) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({fn, dev})) return cudaSuccess;
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem)) != cudaSuccess)
    return e;
  if (nonportable_cluster &&
      (e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
    return e;
  done.insert({fn, dev});
  return cudaSuccess;
}

static unsigned long long g_launches = 0;
void note_launch(unsigned n) { __atomic_fetch_add(&g_launches, (unsigned long long)n, __ATOMIC_RELAXED); }
unsigned long long launch_count() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }
static unsigned long long g_simt_gemms = 0;
void note_simt_gemm() { __atomic_fetch_add(&g_simt_gemms, 1ull, __ATOMIC_RELAXED); }
unsigned long long simt_gemm_count() { return __atomic_load_n(&g_simt_gemms, __ATOMIC_RELAXED); }

cudaError_t gemm_simt_f32(const GemmDesc<float>& g, Round rnd, cudaStream_t s) {
  switch (rnd) {
    case Round::TF32: return launch_gemm<float, Round::TF32>(g, s);
    case Round::BF16: return launch_gemm<float, Round::BF16>(g, s);
    default: return launch_gemm<float, Round::None>(g, s);
  }
}

cudaError_t gemm_simt_f64(const GemmDesc<double>& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (g.zsplit > 1) return launch_gemm<double, Round::None>(g, s);
  dim3 grid((g.N + 15) / 16, (g.M + 15) / 16);
  k_gemm_t16<double><<<grid, 256, 0, s>>>(g);
  note_launch();
  return cudaGetLastError();
}

cudaError_t gemm_small_f32(const GemmDesc<float>& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (g.zsplit > 1) return launch_gemm<float, Round::None>(g, s);
  dim3 grid((g.N + 15) / 16, (g.M + 15) / 16);
  if (g.K <= kT16MaxK) {
    k_gemm_t16_wholek<<<grid, 256, 0, s>>>(g);
  } else {
    k_gemm_t16<float><<<grid, 256, 0, s>>>(g);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t reduce_splitk_f64(const float* part, int nsplit, long long zstride, int n, int ldp, double* out, int ldo,
                              int symmetrize, int* flags, cudaStream_t s, float* out32, double* dscale) {
  long long tot = (long long)n * n;
  if (tot == 0) return cudaSuccess;
  if (dscale && symmetrize == 1) return cudaErrorInvalidValue;  // scaling reads the reduced diagonal: modes 0 and 2
  if (dscale) {
    k_diag_scale<<<(n + 127) / 128, 128, 0, s>>>(part, nsplit, zstride, n, ldp, dscale);
    note_launch();
  }
  k_reduce_splitk<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, nsplit, zstride, n, ldp, out, ldo, symmetrize,
                                                                  out32, flags, dscale);
  note_launch();
  if (symmetrize == 1) {
    k_symmetrize<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(out, n, ldo, out32);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t transpose_f32(const float* in, long long ldi, int rows, int cols, float* out, long long ldo,
                          cudaStream_t s, const double* rdiv) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  k_transpose<<<grid, dim3(32, 8), 0, s>>>(in, ldi, rows, cols, out, ldo, rdiv);
  note_launch();
  return cudaGetLastError();
}

cudaError_t pack_rows_f32(const float* src, long long lds, int rows, int cols, float* dst, long long ldd,
                          cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const long long total = (long long)rows * (ldd >> 2);
  const long long blocks = std::min<long long>((total + 255) / 256, 152LL * 16);
  k_pack_rows<<<(unsigned)blocks, 256, 0, s>>>(src, lds, rows, cols, dst, ldd);
  note_launch();
  return cudaGetLastError();
}

cudaError_t to_bf16_f32(const float* src, long long lds, int rows, int cols, void* dst, long long ldd, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const long long total = (long long)rows * (ldd / 8);
  const long long blocks = std::min<long long>((total + 255) / 256, 152LL * 16);
  k_to_bf16<<<(unsigned)blocks, 256, 0, s>>>(src, lds, rows, cols, static_cast<uint4*>(dst), ldd / 8);
  note_launch();
  return cudaGetLastError();
}

cudaError_t im2col_f32(const float* x, int c, int h, int w, int kh, int kw, int sh, int sw, int ph, int pw, int i0,
                       int ns, int append_one, float scale, float* X, long long ldx, cudaStream_t s) {
  const int ho = (h + 2 * ph - kh) / sh + 1, wo = (w + 2 * pw - kw) / sw + 1;
  const int d = c * kh * kw + (append_one ? 1 : 0);
  if (d <= 0 || ldx <= 0) return cudaSuccess;
  dim3 grid((unsigned)((ldx + 255) / 256), (unsigned)d);
  k_im2col<<<grid, 256, 0, s>>>(x, c, h, w, kh, kw, sh, sw, ph, pw, ho, wo, i0, ns, append_one, scale, X, ldx);
  note_launch();
  return cudaGetLastError();
}

cudaError_t rows_to_cols_f32(const float* A, long long lda, int n, int cols, int append_one, float scale, float* X,
                             long long ldx, cudaStream_t s) {
  const int d = cols + append_one;
  if (d <= 0 || ldx <= 0) return cudaSuccess;
  dim3 grid((unsigned)((ldx + 31) / 32), (unsigned)((d + 31) / 32));
  k_rows_to_cols<<<grid, dim3(32, 8), 0, s>>>(A, lda, n, cols, append_one, scale, X, ldx);
  note_launch();
  return cudaGetLastError();
}

cudaError_t convert_f32_to_f64(const float* in, long long ldi, int rows, int cols, double* out, long long ldo,
                               int* flags, cudaStream_t s) {
  long long tot = (long long)rows * cols;
  if (tot == 0) return cudaSuccess;
  k_convert<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(in, ldi, rows, cols, out, ldo, flags);
  note_launch();
  return cudaGetLastError();
}

}  // namespace kfac
