// Internal declarations shared by the CUDA translation units of libkfac.
// Row-major storage everywhere; "ld" is the row stride in elements.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/kfac.h"

namespace kfac {

// Largest dynamic shared memory a kernel here requests: the 227 KB opt-in limit
// minus 1 KB kept for static shared variables.
constexpr int kSmemOptin = 227 * 1024 - 1024;

// Largest sketch width k = rank + oversample (and largest factor diagonalised
// directly when k >= d): the FP64 Cholesky keeps the k x k Gram and the
// Jacobi keeps its column blocks in the shared memory of a 16-CTA cluster.
constexpr int kMaxSketch = 576;

// Process-wide count of kernel launches issued by this library.
void note_launch(unsigned n = 1);
unsigned long long launch_count();
// Process-wide count of products that gemm_f32 sent to the SIMT kernel
// instead of the tensor cores (K > 0; see kfac_simt_gemm_count).
void note_simt_gemm();
unsigned long long simt_gemm_count();

// Device-side counters (see kfac_stats_read): sweeps, solves, Cholesky, retries.
enum { STAT_SWEEPS = 0, STAT_EIG_SOLVES = 1, STAT_CHOL = 2, STAT_CHOL_RETRY = 3, STAT_COUNT = 4 };

// Device-side status word: kernels OR KFAC_FLAG_* bits into it.
// Asynchronous 4-byte global -> shared copy (zero-filled when !valid). A loop
// of plain loads feeding shared memory waits out the L2 latency (~1000 cycles
// for a far-die hit) once per iteration; these copies are all in flight at
// once and cp_async_wait_all() waits for them together.
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src, bool valid) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(gmem_src), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void raise_flag(int* flags, int bit) {
  if (flags) atomicOr(flags, bit);
}

enum class Round { None = 0, TF32 = 1, BF16 = 2 };

// Operand rounding applied by the SIMT fallback so that its numerics follow the
// selected tensor-core precision (TF32 keeps the top 10 mantissa bits, BF16 rounds
// to nearest even at 7 mantissa bits).
__device__ __forceinline__ float round_operand(float x, Round r) {
  if (r == Round::TF32) return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  if (r == Round::BF16) {
    unsigned u = __float_as_uint(x);
    if ((u & 0x7F800000u) == 0x7F800000u) return x;  // Inf/NaN unchanged
    u += 0x7FFFu + ((u >> 16) & 1u);
    return __uint_as_float(u & 0xFFFF0000u);
  }
  return x;
}

// Generic strided GEMM description: D(m, n) = alpha * rowscale[m] * colscale[n] *
// sum_k A(m, k) B(n, k) + beta * C0(m, n), with A(m, k) = A[m*sam + k*sak] and
// B(n, k) = B[n*sbn + k*sbk]. D(m, n) is D[m*ldd + n], or D[n*ldd + m] with
// d_trans; C0 likewise with c0_trans. sym (M == N, A B^T symmetric): only
// elements with m <= n are computed and each is also written at (n, m), so the
// result is exactly symmetric. When zsplit > 1 the K range is cut into zsplit
// chunks (kchunk a multiple of 32) and chunk z writes its raw partial sums to
// D + z*zstride in D's layout (alpha, scales, beta ignored); the caller reduces
// them. ws (ws_floats floats, optional) lets the dispatcher split K by itself.
template <typename T>
struct GemmDesc {
  int M, N, K;
  const T* A;
  long long sam, sak;
  const T* B;
  long long sbn, sbk;
  T* D;
  long long ldd;
  const T* C0;
  long long ldc;
  T alpha, beta;
  const T* rowscale;
  const T* colscale;
  int zsplit;
  int kchunk;
  long long zstride;
  int d_trans;
  int c0_trans;
  int sym;
  T* ws;
  long long ws_floats;
  int* flags;  // device status word for bounded-wait timeouts (may be null)
  long long wait_cycles;  // limit of the tensor-core kernels' waits on each other's progress (0: default)
  int split_target;       // split K of a product with few tiles up to this many CTAs (0: 152, < 0: never)
  int ab_bf16;            // A and B point to BF16 data (K-major, strides in elements; tensor cores only)
  const T* A_lo;          // FP32 tensor-core products: precomputed 3xTF32 tails of A / B (row strides
  const T* B_lo;          //   ld_alo / ld_blo, 0 = the operand's), or null (the kernel forms them per tile)
  long long ld_alo, ld_blo;
};

// Default limit of a tensor-core kernel's wait for another role's progress:
// ~2 s at 2 GHz, far beyond any legitimate wait (KFAC_OPT_WAIT_CYCLES).
constexpr long long kDefaultWaitCycles = 4000000000LL;

// ---- launchers (host) --------------------------------------------------------
cudaError_t gemm_simt_f32(const GemmDesc<float>& g, Round rnd, cudaStream_t s);
cudaError_t gemm_simt_f64(const GemmDesc<double>& g, cudaStream_t s);
// Kernel attributes belong to a kernel on one device: set the dynamic shared
// memory limit (and, for cluster kernels, non-portable cluster sizes) once per
// kernel and device, on the current device.
cudaError_t set_kernel_attrs_once(const void* fn, int max_dyn_smem, bool nonportable_cluster);

// FP32 product with 16 x 16 output tiles (plain FP32 FMA), for k x k matrices.
cudaError_t gemm_small_f32(const GemmDesc<float>& g, cudaStream_t s);
// out[i, j] = sum_z part[z][i, j] in FP64 (n x n), symmetrised as (S + S^T) / 2
// with symmetrize = 1, or (symmetrize = 2) from partials that hold only the
// upper triangle i <= j, mirrored. part has row stride ldp and z stride zstride.
// out32 (optional): an FP32 copy of the result, n x n dense. dscale (optional,
// symmetrize 0 or 2): the result is column-scaled, out_ij = S_ij / (d_i d_j)
// with d_i = sqrt(S_ii) (1 where S_ii is not positive and finite), and
// dscale[i] = d_i.
cudaError_t reduce_splitk_f64(const float* part, int nsplit, long long zstride, int n, int ldp, double* out,
                              int ldo, int symmetrize, int* flags, cudaStream_t s, float* out32 = nullptr,
                              double* dscale = nullptr);
// out (cols x rows) = in^T; with rdiv, row r of in is divided by rdiv[r] first.
cudaError_t transpose_f32(const float* in, long long ldi, int rows, int cols, float* out, long long ldo,
                          cudaStream_t s, const double* rdiv = nullptr);
// Columns j0 .. j0 + ncols - 1 of the seeded d x k Gaussian test matrix (the
// generator kfac_draw_omega documents): out (d x ncols, row stride ld) or, with
// trans, its transpose (ncols x d, row stride ld).
cudaError_t draw_omega_f32(int d, int k, unsigned long long seed, int j0, int ncols, float* out, long long ld,
                           bool trans, cudaStream_t s);
cudaError_t convert_f32_to_f64(const float* in, long long ldi, int rows, int cols, double* out, long long ldo,
                               int* flags, cudaStream_t s);
// dst (rows x cols, row stride ldd: a multiple of 4 floats, 16-byte aligned
// base) <- src (any row stride lds); the pad columns are zeroed. Gives the
// tensor-core kernels (whose TMA loads need 16-byte row strides) a copy of an
// operand whose rows are not 16-byte aligned.
cudaError_t pack_rows_f32(const float* src, long long lds, int rows, int cols, float* dst, long long ldd,
                          cudaStream_t s);
// X (d x ldx, d = cols + append_one, ldx >= n) <- scale * A^T for a row-major
// batch A (n x cols), plus a last row of ones when append_one; pad columns zeroed.
cudaError_t rows_to_cols_f32(const float* A, long long lda, int n, int cols, int append_one, float scale, float* X,
                             long long ldx, cudaStream_t s);
// Patch matrix (d x ldx, d = c kh kw + append_one) of samples [i0, i0 + ns) of
// an NCHW convolution input: column (sample, output position), row (channel,
// kernel row, kernel column), zero padding, times `scale`; pad columns zeroed.
cudaError_t im2col_f32(const float* x, int c, int h, int w, int kh, int kw, int sh, int sw, int ph, int pw, int i0,
                       int ns, int append_one, float scale, float* X, long long ldx, cudaStream_t s);
// dst (rows x cols BF16, row stride ldd a multiple of 8, 16-byte aligned) <-
// src (FP32, row stride lds) rounded to nearest even; pad columns zeroed.
cudaError_t to_bf16_f32(const float* src, long long lds, int rows, int cols, void* dst, long long ldd, cudaStream_t s);
// True when TMA can read a row-major FP32 matrix at p with row stride ld as is
// (16-byte aligned base and row stride).
inline bool tma_rows_ok(const void* p, long long ld) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0 && (ld & 3) == 0;
}

// Cholesky of (G + shift I) on a thread-block cluster, factorised in FP64
// (fp64) or FP32 from the FP64 Gram G; writes the lower factor L as FP32 (k x k
// row-major, upper part zero). shift = shift_rel * trace(G) for shift_rel > 0,
// |shift_rel| * trace(G) / k for shift_rel < 0. A pivot below a floor tied to
// the FP32 rounding level is raised to it (flag CHOL_SHIFTED); a non-finite
// pivot retries with a growing shift (bounded) and then fails (CHOL_FAILED).
// shift_out (optional, device) receives the shift the successful attempt used.
// G32 (optional, row stride ld32): an FP32 copy of G that the FP32 path reads
// instead of converting G (a conversion runs on the FP64 pipe).
// nc_pref: cluster size of the multi-CTA kernel (0 = one CTA per 16 rows, at
// most 16; raised to the fewest CTAs whose shared memory holds the rows).
// panel: its panel width, 16 or 32 (halved while the shared memory overflows).
cudaError_t chol_cluster(const double* G, int k, double shift_rel, bool fp64, float* L32, int* flags,
                         unsigned long long* stats, cudaStream_t s, double* shift_out = nullptr,
                         const float* G32 = nullptr, long long ld32 = 0, int nc_pref = 0, int panel = 16);

// Blocked FP32 Cholesky (the same contract as chol_cluster's FP32 path) for
// k above the one-CTA kernel's limit: one-CTA factorisations of diagonal
// blocks, triangular solves and tensor-core rank updates between them. G32 (row
// stride ld32) is required; ws: chol_blocked_ws_bytes(k) bytes of device
// workspace. k within the one-CTA limit goes to chol_cluster.
// Row i of the lower factor L32 (k x k, dense) times dscale[i]: the factor of
// a column-scaled Gram (reduce_splitk_f64's dscale) back to the Gram's scale.
cudaError_t factor_unscale(float* L32, int k, const double* dscale, cudaStream_t s);
size_t chol_blocked_ws_bytes(int k);
cudaError_t chol_blocked(const double* G, const float* G32, long long ld32, int k, double shift_rel, float* L32,
                         int* flags, unsigned long long* stats, cudaStream_t s, double* shift_out, void* ws,
                         long long wait_cycles);

// Qt = L^-1 Yt for lower-triangular FP32 L (k x k) and Yt (k x d, row stride ldy).
// dinv_ws: trsm_ws_floats(k) floats of workspace (L packed by 32-row block rows
// with inverted diagonal blocks, or the block inverses alone for large k).
inline size_t trsm_ws_floats(int k) {
  const size_t T = (size_t)(k + 31) / 32;
  return T * 1024 > 512 * T * (T + 1) ? T * 1024 : 512 * T * (T + 1);
}
// qlo (optional, row stride ldlo): the TF32 tails of Qt (tf32_tail) stored
// beside it, the tail plane the next 3xTF32 product of Qt reads.
cudaError_t trsm_lower_f32(const float* L, int k, const float* Yt, long long ldy, float* Qt, long long ldq, int d,
                           float* dinv_ws, cudaStream_t s, float* qlo = nullptr, long long ldlo = 0);
// The same solve blocked over the blocked Cholesky's diagonal blocks, the
// off-diagonal work as FP32-accurate tensor-core products (for k above the
// shared-memory solve's range: trsm_blocked_used(k)). ws: trsm_blocked_ws_bytes
// (k, d) bytes of device workspace; Yt and Qt must not overlap.
bool trsm_blocked_used(int k);
size_t trsm_blocked_ws_bytes(int k, int d);
cudaError_t trsm_blocked(const float* L, int k, const float* Yt, long long ldy, float* Qt, long long ldq, int d,
                         void* ws, int* flags, long long wait_cycles, cudaStream_t s);
// The same solve through the explicit inverse: L^-1 by solving the identity,
// then Qt = (Yt^T L^-T)^T as one FP32-accurate tensor-core product. ws:
// trsm_inverse_ws_bytes(k, d) bytes of device workspace. dscale (optional):
// L is the factor of a column-scaled Gram and the solve uses D L (row i of L
// times dscale[i]): Qt = L^-1 (D^-1 Yt), the rows of Yt divided by dscale as
// they are transposed for the product (L^-1 itself is not scaled, so it keeps
// the magnitude it has without the scaling).
size_t trsm_inverse_ws_bytes(int k, int d);
cudaError_t trsm_inverse(const float* L, int k, const float* Yt, long long ldy, float* Qt, long long ldq, int d,
                         void* ws, int* flags, long long wait_cycles, cudaStream_t s, const double* dscale = nullptr);

// FP32 one-sided Jacobi on chol(C + s I) over a thread-block cluster: writes X
// (k x k FP64, column j = unit eigenvector) and lam (k, unsorted). gscratch:
// eig_scratch_floats(k) floats (the Cholesky factor and the shift it used).
// (the factor, the shift, then the blocked Cholesky's workspace 256-byte aligned)
inline size_t eig_scratch_head_floats(int k) { return ((((size_t)k * k + 1) & ~(size_t)1) + 4 + 63) & ~(size_t)63; }
inline size_t eig_scratch_floats(int k) { return eig_scratch_head_floats(k) + (chol_blocked_ws_bytes(k) + 3) / 4; }
// stop_tol > 0 ends the sweeps after one whose largest pair cosine was below it.
// chol_blocked: factor C + sI by chol_blocked (k above the one-CTA limit, C32
// given) instead of the cluster kernel.
cudaError_t eig_jacobi_f32(const double* C, int k, double shift_rel, int max_sweeps, float tol, float stop_tol,
                           double* X, double* lam, float* gscratch, int* flags, unsigned long long* stats,
                           cudaStream_t s, const float* C32 = nullptr, long long ld32 = 0, int chol_nc = 0,
                           int chol_panel = 16, int chol_blocked = 0, long long wait_cycles = 0);

// One-sided Jacobi on the columns of the k x k FP32 matrix held in gscratch
// (row-major; the factor eig_jacobi_f32 writes there), with the device scalar
// `shift`: writes X (column j = unit column j after the rotations) and
// lam_j = |w_j|^2 - shift (unsorted). full = 0 reads only the lower triangle
// (a Cholesky factor), 1 the whole matrix.
cudaError_t jacobi_columns(int k, int max_sweeps, float tol, float stop_tol, double* X, double* lam, float* gscratch,
                           const double* shift, int* flags, unsigned long long* stats, cudaStream_t s, int full);
// Thin SVD of a k x k FP32 matrix W (row-major, dense) by one-sided Jacobi:
// W = U diag(sigma) V^T; writes X = U (column j = left singular vector j) and
// lam_j = sigma_j^2 (unsorted). gscratch: eig_scratch_floats(k) floats.
cudaError_t svd_jacobi_f32(const float* W32, int k, int max_sweeps, float tol, float stop_tol, double* X, double* lam,
                           float* gscratch, int* flags, unsigned long long* stats, cudaStream_t s);

// G <- (3 I - G) / 2 in place (k x k FP64): one Newton-Schulz step towards
// G^-1/2 for a Gram G = Q^T Q near I, so Q (3I - G)/2 is orthonormal to
// second order in ||G - I||.
cudaError_t polish_factor(double* G, int k, cudaStream_t s);
cudaError_t convert_f64_to_f32(const double* in, long long n, float* out, cudaStream_t s);

// One FP64 refinement step (Ogita-Aishima) of eigenpairs (X, lam) of C.
// Workspace: eig_refine_doubles(k) doubles. X and lam are updated in place.
inline size_t eig_refine_doubles(int k) { return 5 * (size_t)k * k + 3 * 128; }
cudaError_t eig_refine_f64(const double* C, int k, double* X, double* lam, double* work, int* flags,
                           cudaStream_t s);
// The same step with FP32 k x k products (C32 = FP32 copy of C, row stride
// ldc32): their rounding (~6e-8 of ||C||) is at the accuracy C itself carries.
// w32: eig_refine_floats(k) floats; part: 3 * 128 doubles. The FP32 work
// matrices have the row stride ref_ld(k), so their products (from k = 128 up)
// run on the tensor cores.
inline long long ref_ld(int k) { return ((long long)k + 3) / 4 * 4; }
inline size_t eig_refine_floats(int k) { return 8 * (size_t)k * ref_ld(k); }
// Floats of w32 the basis polish uses (E, P, Q and a padded copy of C32).
inline size_t polish_floats(int k) { return 4 * (size_t)k * ref_ld(k); }
cudaError_t eig_refine_f32(const float* C32, long long ldc32, int k, double* X, double* lam, float* w32, double* part,
                           int* flags, cudaStream_t s);
// Basis polish in FP32 products: with E = G - I (G = Q^T Q, FP64) and
// M = I - E/2 = (3I - G)/2, C <- M C M (C32, row stride k, updated too) keeps
// E (row stride ref_ld(k)) at the start of w32 (polish_floats(k) floats) for
// polish_vectors_f32, which applies X <- M X.
cudaError_t polish_projected_f32(const double* G, double* C, float* C32, int k, float* w32, cudaStream_t s);
cudaError_t polish_vectors_f32(double* X, int k, float* w32, cudaStream_t s);
// E = G - I (FP32, k x k, row stride ref_ld(k)) at the start of w32, for polish_vectors_f32.
cudaError_t polish_E_f32(const double* G, int k, float* w32, cudaStream_t s);

// Sort eigenpairs descending (stable by index), emit the r leading ones:
// Pt (r x k FP32, row stride ldpt, row t = eigenvector t; optional), D and coef
// (FP32, Eq. (13)), and optionally Uout (k x r into a strided FP32 matrix, for
// the k >= d path).
// singular != 0: lam holds squared singular values; D = sqrt(max(lam, 0)).
cudaError_t eig_select(const double* X, const double* lam, int k, int r, float lambda, float* Pt, long long ldpt,
                       float* D, float* coef, float* Uout, long long ldu, cudaStream_t s, int singular = 0);

// FP32 rounded to TF32 (to nearest, ties away).
__device__ __forceinline__ float tf32_head(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// The tail of x below the TF32 the tensor core reads from an FP32 operand (it
// drops the 13 low mantissa bits), rounded to nearest TF32: x - trunc(x) is
// exact in FP32 and below 2^-10 |x|, so x ~ trunc(x) + tail to 2^-21 |x|,
// without a sign bias. The 3xTF32 products' tail planes hold these values.
__device__ __forceinline__ float tf32_tail(float x) {
  return tf32_head(x - __uint_as_float(__float_as_uint(x) & 0xffffe000u));
}

}  // namespace kfac
