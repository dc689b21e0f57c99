/*
 * kfac.h - C ABI of the GB300 (sm_103a) randomized K-FAC library.
 *
 * The library implements the data-parallel hot path of randomized K-FAC
 * (C. O. Puiu, "Randomized K-FACs: Speeding up K-FAC with Randomized Numerical
 * Linear Algebra", arXiv 2206.15397):
 *   - the exponentially averaged (EA) Kronecker-factor update (Alg. 1, the
 *     forward- and backward-factor EA updates; closed form Eq. (6));
 *   - the randomized low-rank eigendecomposition of a factor (Alg. 3, SREVD,
 *     with the power iterations of Sec. 2.2): Gaussian sketch, power
 *     iterations, orthonormalisation, projected eigenproblem C = Q^T F Q, lift;
 *   - the damped low-rank preconditioner apply (Alg. 4, the M and S updates,
 *     with the low-rank inverse of Eq. (13); Alg. 5 feeds it U~).
 *
 * Conventions shared by every entry point
 *   - Matrices are dense, row-major, FP32, with a leading dimension (ld, in
 *     elements, >= the column count). Every matrix pointer is DEVICE memory of
 *     the context's device, owned by the caller; the library never frees or
 *     retains it after the call's work has completed on the stream.
 *   - Calls are stream-ordered and asynchronous on the context's stream.
 *     Argument errors are detected on the host and returned synchronously
 *     before anything is enqueued. Numerical conditions met on the device
 *     (Cholesky breakdown, non-convergence, non-finite values) are recorded in
 *     a device status word and returned by kfac_get_status().
 *   - The library owns one workspace per context (device memory it allocates
 *     itself and grows on demand; kfac_reserve() pre-sizes it, which a caller
 *     that captures calls into a CUDA graph must do first).
 *   - A context is not thread-safe: one host thread at a time.
 *   - No call aborts, traps or prints.
 */
#ifndef KFAC_H_
#define KFAC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define KFAC_API __attribute__((visibility("default")))
#else
#define KFAC_API
#endif

typedef enum {
  KFAC_OK = 0,
  KFAC_ERR_INVALID_ARG = 1,  /* bad size, null pointer, ld too small, ...      */
  KFAC_ERR_CUDA = 2,         /* a CUDA runtime call failed                      */
  KFAC_ERR_OOM = 3,          /* workspace allocation failed                     */
  KFAC_ERR_CHOLESKY = 4,     /* Gram Cholesky broke down even after shifting    */
  KFAC_ERR_NOCONVERGE = 5,   /* Jacobi sweep limit reached                      */
  KFAC_ERR_NONFINITE = 6,    /* NaN/Inf met in an input or an intermediate      */
  KFAC_ERR_TIMEOUT = 7,      /* a bounded device-side wait gave up              */
  KFAC_ERR_UNSUPPORTED = 8,  /* valid request this build does not implement     */
  KFAC_ERR_TOO_LARGE = 9     /* request exceeds a fixed-size static scratch area */
} kfac_status;

/* Arithmetic of the large GEMMs (EA SYRK, sketch / power / projection, apply).
 * The orthonormalisation and the eigensolve keep their own precision in every
 * mode: FP32-accurate Grams summed with compensation into FP64, FP32 Cholesky,
 * FP32 Jacobi and an eigen-refinement with FP32 products and FP64 carriers
 * (KFAC_OPT_CHOLQR_FP32_PASSES and KFAC_OPT_EIG_REFINE_FP64 select FP64). */
typedef enum {
  KFAC_PREC_FP32 = 0,  /* FP32-accurate products (3xTF32 split on tensor cores)  */
  KFAC_PREC_TF32 = 1,  /* single-pass TF32 tensor-core products, FP32 accumulate */
  KFAC_PREC_BF16 = 2   /* BF16 operands on tensor cores, FP32 accumulate         */
} kfac_precision;

/* Device status bits accumulated since the last kfac_get_status(). */
enum {
  KFAC_FLAG_CHOL_SHIFTED = 1 << 0,   /* a Gram Cholesky needed an extra diagonal shift  */
  KFAC_FLAG_CHOL_FAILED = 1 << 1,    /* ... and still broke down                       */
  KFAC_FLAG_EIG_NOCONV = 1 << 2,     /* Jacobi hit its sweep cap                       */
  KFAC_FLAG_NONFINITE = 1 << 3,      /* NaN/Inf seen                                   */
  KFAC_FLAG_EIG_SHIFTED = 1 << 4,    /* eigensolver needed a larger PD shift           */
  KFAC_FLAG_TIMEOUT = 1 << 5         /* a bounded device wait expired                  */
};

typedef struct kfac_ctx kfac_ctx;

/* Library version (major * 10000 + minor * 100 + patch). */
KFAC_API int kfac_version(void);

/* Static, human-readable name of a status code. Never NULL. */
KFAC_API const char* kfac_status_string(kfac_status st);

/* Create a context bound to CUDA device `device` and stream `stream` (a
 * cudaStream_t passed as void*; NULL = the legacy default stream). *out
 * receives an opaque handle owned by the caller (free with kfac_destroy). */
KFAC_API kfac_status kfac_create(kfac_ctx** out, int device, void* stream);

/* Synchronise the context's stream and release its workspace and handle. */
KFAC_API kfac_status kfac_destroy(kfac_ctx* ctx);

/* Re-bind the context to another stream of the same device. */
KFAC_API kfac_status kfac_set_stream(kfac_ctx* ctx, void* stream);

/* Pre-size the workspace for calls with factor dimension <= d_max, sketch
 * width k = rank + oversample <= k_max and preconditioned matrices of at most
 * mn_max elements (0 = none). Needed before graph capture; optional otherwise. */
KFAC_API kfac_status kfac_reserve(kfac_ctx* ctx, int d_max, int k_max, int64_t mn_max);

/* EA K-factor update, Alg. 1 (forward / backward factor EA updates):
 *     F <- rho * F + (1 - rho) / n * X X^T
 * X: d x n batch matrix (one column per sample, row stride ldx >= n).
 * F: d x d symmetric factor, in/out (row stride ldf >= d); both triangles are
 *    written, and the result is exactly symmetric.
 * prec selects the product arithmetic (FP32 / TF32 / BF16 operands).
 * The 1/n normalisation reads Alg. 1's A A^T as the batch mean. */
KFAC_API kfac_status kfac_ea_update(kfac_ctx* ctx, int d, int n, const float* X, int ldx, float rho,
                                    kfac_precision prec, float* F, int ldf);

/* The same EA update from a batch in the layout a layer sees it: A is n x cols
 * row-major (one sample per row, row stride lda >= cols), e.g. a linear
 * layer's input activations or its output gradients. The factor is
 * d x d with d = cols + append_one: with append_one != 0 the homogeneous
 * coordinate 1 is appended last to every sample (the bias column of Mat(g)).
 * Every sample is multiplied by `scale` first (e.g. the batch size for the
 * gradients of a batch-mean loss, so that they are per-sample gradients):
 *     F <- rho F + (1 - rho) / n * scale^2 * Abar^T Abar,   Abar = [A, 1].
 * The batch is transposed into the context workspace (one kernel) and the
 * product runs as kfac_ea_update. */
KFAC_API kfac_status kfac_ea_update_rows(kfac_ctx* ctx, int n, int cols, const float* A, int lda, int append_one,
                                         float scale, float rho, kfac_precision prec, float* F, int ldf);

/* EA update of a convolutional layer's K-factor from patch statistics (the
 * conv K-factors of Eq. (4), which the paper takes from KFC): the columns of
 * the batch matrix are the layer's input patches at every sample and output
 * position,
 *     F <- rho F + (1 - rho) / (n ho wo) * sum_{i, oy, ox} p p^T,
 *     p[(ch kh + r) kw + t] = scale * x[i, ch, oy sh + r - ph, ox sw + t - pw]
 * (zero outside the image; with append_one the entry `scale` is appended last
 * for the bias), so F is d x d with d = c kh kw + append_one, ordered as a
 * PyTorch conv weight (C_out, C_in, kh, kw) flattens per output channel.
 * x: n x c x h x w input activations (NCHW, contiguous, device memory);
 * ho = (h + 2 ph - kh) / sh + 1, wo likewise. The backward factor of the same
 * layer is this call on the output gradients (n x C_out x ho x wo) with a 1 x 1
 * kernel, stride 1, no padding, append_one 0 and scale = n for a batch-mean
 * loss. The patch matrix is built in the context workspace in chunks of whole
 * samples of at most KFAC_OPT_CONV_CHUNK floats, each chunk accumulated by the
 * tensor-core SYRK of kfac_ea_update. */
KFAC_API kfac_status kfac_ea_update_conv(kfac_ctx* ctx, int n, int c, int h, int w, const float* x, int kh, int kw,
                                         int stride_h, int stride_w, int pad_h, int pad_w, int append_one, float scale,
                                         float rho, kfac_precision prec, float* F, int ldf);

/* One factor of a grouped EA update (arguments as kfac_ea_update). */
typedef struct {
  int d, n;
  const float* X;
  int ldx;
  float rho;
  kfac_precision prec;
  float* F;
  int ldf;
} kfac_ea_desc;

/* kfac_ea_update for `count` factors (every layer's forward and backward
 * factor, Alg. 1), enqueued on up to KFAC_OPT_GROUP_STREAMS streams forked from the context stream
 * (event fork/join, graph-capturable; factors taken largest first, each on the
 * stream with the least work so far). A batch matrix whose base or row stride
 * is not 16-byte aligned is first copied into the workspace with a padded
 * stride (so that the product runs on the tensor cores); a call that does this
 * under graph capture needs the workspace sized by an earlier call with the same
 * shapes. All descriptors are checked before anything is enqueued; factors must
 * not alias each other. */
KFAC_API kfac_status kfac_ea_update_grouped(kfac_ctx* ctx, int count, const kfac_ea_desc* descs);

/* Randomized low-rank eigendecomposition + damping coefficients of one
 * symmetric PSD factor F (d x d), Alg. 3 with power iterations (Sec. 2.2):
 *     Y = F Omega; Q = orth(Y); repeat power_iters times: Q = orth(F Q);
 *     C = Q^T F Q; C = P diag(L) P^T (descending); U = Q P[:, :r]; D = L[:r];
 *     coef_i = 1/(max(D_i, 0) + lambda) - 1/lambda            (Eq. (13))
 * k = rank + oversample columns are sketched; r = min(rank, d) are returned.
 * When k >= d the factor is diagonalised directly (Q = I). The sketch width
 * (or d on that direct path) is limited to 576: larger requests return
 * KFAC_ERR_UNSUPPORTED.
 * omega: d x k Gaussian test matrix (row stride ldo >= k), drawn by the caller;
 *        or NULL: the library draws the matrix kfac_draw_omega gives for `seed`
 *        on the device, straight into the transposed layout the sketch reads
 *        (no copy in, no transpose). Ignored when k >= d (may be NULL).
 * seed:  the generator key when omega is NULL (ignored otherwise).
 * U: d x r output (row stride ldu >= r); D, coef: r outputs.
 * F must hold the full symmetric matrix (both triangles are read; F is not
 * modified). power_iters counts extra products F Q, each followed by a fresh
 * orthonormalisation, so the basis spans F^(power_iters + 1) Omega. */
KFAC_API kfac_status kfac_rsvd_invert(kfac_ctx* ctx, int d, const float* F, int ldf, int rank, int oversample,
                                      int power_iters, float lambda, const float* omega, int ldo,
                                      unsigned long long seed, kfac_precision prec, float* U, int ldu, float* D,
                                      float* coef);

/* The library's Gaussian test matrix for a seed (Omega of Alg. 2 / Alg. 3,
 * i.i.d. N(0, 1) entries), written to omega (d x k, row stride ldo >= k) on the
 * context stream. Element (i, j) is value e = i*k + j of one counter-based
 * stream, Philox4x32 with 10 rounds (Salmon, Moraes, Dror and Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11) keyed by the seed's low and high
 * 32-bit halves:
 *   block b = floor(e / 4) has the counter (b mod 2^32, floor(b / 2^32), 0, 1)
 *   and gives the words w0..w3; a word w maps to (floor(w / 512) + 1/2) / 2^23
 *   in (0, 1) (exact in FP32); values 4b and 4b+1 are rho cos(2 pi v) and rho sin(2 pi v) with
 *   rho = sqrt(-2 ln u), u from w0 and v from w1 (Box-Muller); values 4b+2 and
 *   4b+3 the same from w2 and w3.
 * Evaluated in FP32 (logf, sqrtf, sincospif): each value is within a few units
 * in the last place of the same formula evaluated exactly. kfac_rsvd_invert and
 * the grouped inversion draw this matrix when their omega is NULL. Returns
 * KFAC_ERR_INVALID_ARG for d or k < 1, a NULL omega or ldo < k. */
KFAC_API kfac_status kfac_draw_omega(kfac_ctx* ctx, int d, int k, unsigned long long seed, float* omega, int ldo);

/* One factor of a grouped inversion: the arguments of kfac_rsvd_invert. */
typedef struct {
  int d;
  const float* F;
  int ldf;
  int rank, oversample, power_iters;
  float lambda;
  const float* omega;
  int ldo;
  kfac_precision prec;
  float* U;
  int ldu;
  float* D;
  float* coef;
  unsigned long long seed; /* generator key when omega is NULL (kfac_draw_omega) */
} kfac_invert_desc;

/* kfac_rsvd_invert for `count` independent factors (the per-layer loop of
 * Alg. 4/5). The factors' pipelines are enqueued on up to KFAC_OPT_GROUP_STREAMS streams forked
 * from the context stream (event fork/join, graph-capturable; the costliest
 * factor first, each on the stream with the least estimated work so far), each
 * stream with its own workspace slice, so the latency-bound small-matrix steps of different
 * factors overlap on the GPU. Arguments of every descriptor are checked before
 * anything is enqueued; the host array may be reused once the call returns. */
KFAC_API kfac_status kfac_rsvd_invert_grouped(kfac_ctx* ctx, int count, const kfac_invert_desc* descs);

/* Damped Kronecker preconditioner apply, Alg. 4 (M and S updates) with Eq. (13):
 *     M = J U_a diag(coef_a) U_a^T + J / lambda
 *     S = U_g diag(coef_g) U_g^T M + M / lambda
 * i.e. S = (U_g D_g U_g^T + lambda I)^-1 J (U_a D_a U_a^T + lambda I)^-1.
 * J: d_g x d_a gradient matrix Mat(g) (row stride ldj >= d_a; bias gradient in
 *    the last column when the layer has a bias).
 * U_a: d_a x r_a (ld_ua >= r_a), coef_a: r_a; U_g: d_g x r_g (ld_ug >= r_g),
 * coef_g: r_g. r_a or r_g may be 0. lambda must equal the value given to
 * kfac_rsvd_invert. S: d_g x d_a output (lds >= d_a); S must not alias J. */
KFAC_API kfac_status kfac_precondition(kfac_ctx* ctx, int d_g, int d_a, const float* J, int ldj,
                                       const float* U_a, int ld_ua, const float* coef_a, int r_a,
                                       const float* U_g, int ld_ug, const float* coef_g, int r_g,
                                       float lambda, kfac_precision prec, float* S, int lds);

/* One layer of a grouped preconditioner apply (arguments as kfac_precondition). */
typedef struct {
  int d_g, d_a;
  const float* J;
  int ldj;
  const float* U_a;
  int ld_ua;
  const float* coef_a;
  int r_a;
  const float* U_g;
  int ld_ug;
  const float* coef_g;
  int r_g;
  float lambda;
  kfac_precision prec;
  float* S;
  int lds;
} kfac_precond_desc;

/* kfac_precondition for `count` layers (the per-layer loop of Alg. 4),
 * enqueued on up to KFAC_OPT_GROUP_STREAMS streams forked from the context stream, each stream with
 * its own workspace slice (graph-capturable once kfac_reserve or an earlier
 * call has sized the workspace). All descriptors are checked first. */
KFAC_API kfac_status kfac_precondition_grouped(kfac_ctx* ctx, int count, const kfac_precond_desc* descs);

/* One K-FAC step of a set of layers (Alg. 1: the EA updates of the factors,
 * their inversions by Alg. 3 or Alg. 2, and Alg. 4's apply for every layer),
 * with per-item dependencies instead of a join between the phases. Factor f
 * (0 <= f < n_factors) takes ea[f] (skipped when ea is NULL) and then the
 * inversion inv[f], in turn, on one of up to KFAC_OPT_GROUP_STREAMS streams
 * forked from the context stream (the costliest factors first, each on the
 * least-loaded stream). Layer l (0 <= l < n_layers) takes the apply pre[l] as
 * soon as the inversions of factors layer_factors[2l] and layer_factors[2l+1]
 * (-1: none) have finished, on the stream of the later of the two, so the
 * applies of early layers overlap the inversions still running. pre[l]'s U and
 * coefficient pointers should be those inversions' outputs; the call orders
 * the work, it does not check that. The results are those of
 * kfac_ea_update_grouped + kfac_rsvd_invert_grouped + kfac_precondition_grouped
 * on the same descriptors. All descriptors are checked before anything is
 * enqueued; per-item flags (kfac_get_item_status) are factors 0..n_factors-1
 * then layers. Graph-capturable once an earlier call has sized the workspace. */
KFAC_API kfac_status kfac_step_grouped(kfac_ctx* ctx, int n_factors, const kfac_ea_desc* ea,
                                       const kfac_invert_desc* inv, int n_layers, const kfac_precond_desc* pre,
                                       const int* layer_factors);

/* Allocation-free variant of kfac_precondition (the paper has no counterpart:
 * this is a deployment interface). It is for callers that cannot allocate GPU
 * memory at call time: code that runs while a CUDA graph is being captured,
 * runtimes that hand out all device memory up front through their own pool,
 * or processes whose allocator is locked. It needs no kfac_ctx (creating one
 * allocates) and never calls cudaMalloc, cudaFree or any allocating library
 * routine.
 *
 * Same inputs and output as kfac_precondition, with results that agree with it
 * to within rounding (the products are formed in another order: T and the
 * final product read U_a / U_g transposed and T2 reads M through S, so those
 * three run on the SIMT kernel, only M = T U_a^T + J / lambda on the tensor
 * cores), on `stream` (a cudaStream_t as void*; NULL = legacy default stream)
 * of the CURRENT device.
 * The caller's S doubles as the staging area of M. The two thin intermediates
 * T = J U_a diag(coef_a) (d_g x r_a) and T2 = diag(coef_g) U_g^T M
 * (r_g x d_a) take turns in a static device array of KFAC_NOALLOC_SCRATCH_FLOATS
 * floats (8 MiB) that every GPU loading this library holds until the process
 * exits. Requests with max(d_g*r_a, r_g*d_a) > KFAC_NOALLOC_SCRATCH_FLOATS
 * return KFAC_ERR_TOO_LARGE before any work is enqueued.
 *
 * The first call on a device resolves the array's device address for that
 * device (cudaGetSymbolAddress with the device current); make that first call
 * before any stream capture. All calls share the one array and it keeps the
 * previous call's contents (every element read is written first in the same
 * call, so nothing needs clearing); calls whose work overlaps on the GPU (two
 * streams, or two host threads) race on it and must be serialised by the
 * caller. Argument errors return KFAC_ERR_INVALID_ARG; launch errors
 * KFAC_ERR_CUDA. There is no device status word: NaN/Inf propagate to S, and a
 * bounded wait of the tensor-core product that runs out (~2 s; not expected in
 * practice) is not reported by this entry point and leaves S undefined. */
#define KFAC_NOALLOC_SCRATCH_FLOATS (2 * 1024 * 1024)
KFAC_API kfac_status kfac_precondition_noalloc(void* stream, int d_g, int d_a, const float* J, int ldj,
                                               const float* U_a, int ld_ua, const float* coef_a, int r_a,
                                               const float* U_g, int ld_ug, const float* coef_g, int r_g,
                                               float lambda, kfac_precision prec, float* S, int lds);

/* Autotuner of a grouped inversion's schedule on this GPU: the number of
 * streams a grouped call forks (KFAC_OPT_GROUP_STREAMS), the CTA count split-K
 * products may fill (KFAC_OPT_SPLIT_TARGET) and, when a sketch width exceeds
 * the one-CTA Cholesky's 236, the large-order Cholesky: blocked or on a
 * cluster (KFAC_OPT_CHOL_BLOCKED) and, for the cluster kernel, its size and
 * panel width (KFAC_OPT_CHOL_CLUSTER, KFAC_OPT_CHOL_PANEL); the form of the
 * CholeskyQR solves (KFAC_OPT_TRSM_INVERSE) is reported as set. Runs
 * kfac_rsvd_invert_grouped(ctx, count, descs) once plus twice timed (CUDA
 * events on the context stream) per candidate of a coordinate descent from the
 * current settings, writing the descriptors' outputs as a call would, and
 * keeps the fastest settings in the context. cache_path (may be NULL): a text
 * file of earlier results, one line per device name and shape signature (the
 * factors' d, k, power iterations and precision, and the inversion method); a
 * hit is applied without timing, a new result is appended. chosen (may be
 * NULL, 7 ints) receives the streams, cluster size, split target, panel width,
 * blocked flag, solve form and 1 if the result came from the cache. Not during
 * stream capture (it synchronises). */
KFAC_API kfac_status kfac_autotune_invert(kfac_ctx* ctx, int count, const kfac_invert_desc* descs,
                                          const char* cache_path, int* chosen);

/* Synchronise the context's stream, return KFAC_OK or the most severe device
 * condition recorded since the last call (by any entry point, grouped items
 * included), store the raw KFAC_FLAG_* bits in *flags (may be NULL) and clear
 * them, the per-item words of kfac_get_item_status included. */
KFAC_API kfac_status kfac_get_status(kfac_ctx* ctx, int* flags);

/* Per-item attribution of device conditions in grouped calls: item i of a
 * grouped EA update, inversion or apply raises its KFAC_FLAG_* bits in word i
 * of a per-context array, so a breakdown can be traced to its factor or layer.
 * Synchronises the context's stream and stores words 0..count-1 in
 * item_flags (0 for items no grouped call has used); does not clear them.
 * The words accumulate over grouped calls until kfac_get_status clears them,
 * so read them after each grouped call whose items should be told apart. */
KFAC_API kfac_status kfac_get_item_status(kfac_ctx* ctx, int count, int* item_flags);

/* Tunables (defaults in brackets). Returns KFAC_ERR_INVALID_ARG for an unknown
 * option or an out-of-range value. */
typedef enum {
  KFAC_OPT_CHOLQR_PASSES = 0,   /* CholeskyQR passes for the final basis Q [3], 1..6      */
  KFAC_OPT_CHOLQR_SHIFT = 1,    /* first-pass diagonal shift, relative to trace(G) [1e-5] */
  KFAC_OPT_EIG_REFINE = 2,      /* eigen-refinement steps after FP32 Jacobi [1], 0..3    */
  KFAC_OPT_EIG_MAX_SWEEPS = 3,  /* Jacobi sweep cap [40]                                  */
  KFAC_OPT_EIG_TOL = 4,         /* Jacobi pair-orthogonality threshold [2e-6]            */
  KFAC_OPT_CHOLQR_INNER_PASSES = 5, /* passes for a basis that only feeds the next power
                                       iteration [3], 1..6; fewer passes save time but
                                       lose accuracy on ill-conditioned sketches */
  KFAC_OPT_CHOLQR_INNER_FP32 = 8,   /* 1 [default]: every CholeskyQR pass of a basis that
                                       only feeds the next power iteration factors in FP32
                                       (its span, not its orthonormality to FP64 accuracy,
                                       is what the next product needs). 0: inner bases
                                       follow KFAC_OPT_CHOLQR_FP32_PASSES like the final one */
  KFAC_OPT_BASIS_POLISH = 7,        /* 1 [default]: after the final orthonormalisation the
                                       Rayleigh-Ritz step uses Q M, M = (3I - Q^T Q)/2 (one
                                       Newton-Schulz step, applied to the k x k projected
                                       matrix and to the eigenvectors), which restores
                                       orthonormality to second order when the sketch is so
                                       ill-conditioned that FP32-stored CholeskyQR3 leaves
                                       ~1e-4; 0: off */
  KFAC_OPT_CHOLQR_FP32_PASSES = 6,  /* leading passes of every orthonormalisation whose
                                       Cholesky runs in FP32 instead of FP64 [6 = all],
                                       0..6; the last pass of a basis runs in FP64 unless
                                       the value covers every pass. FP32 suffices: the
                                       first, shifted pass only preconditions Y (any
                                       invertible R leaves span(Y R^-1) = span(Y)), each
                                       later pass squares the orthogonality error, and the
                                       basis polish (KFAC_OPT_BASIS_POLISH) squares what is
                                       left */
  KFAC_OPT_EIG_STOP_TOL = 9,        /* [3e-3]: Jacobi also stops after a sweep in which
                                       every pair cosine, taken before its rotation, was <= v;
                                       cyclic Jacobi converges quadratically, so that sweep
                                       leaves them near v^2, and the refinement that follows
                                       squares the remaining error again. 0: sweep until a
                                       sweep rotates no pair (every pair cosine <=
                                       KFAC_OPT_EIG_TOL) */
  KFAC_OPT_CONV_CHUNK = 17,         /* [32 Mi]: floats of one chunk of the patch matrix that
                                       kfac_ea_update_conv builds in the workspace (whole
                                       samples per chunk, at least one) */
  KFAC_OPT_WARM_START = 16,         /* [0]: 1 = subspace iteration across inversions (a variant
                                       beyond the paper): the sketch matrix is [U_prev | omega'],
                                       U_prev being what the call's U buffer holds on entry (the
                                       previous inversion of the same factor, same d and r) and
                                       omega' the first k - r columns of omega (of the seeded
                                       matrix when omega is NULL). The EA factor moves
                                       little between inversions, so C = Q^T F Q starts nearly
                                       diagonal and the Jacobi solve stops after fewer sweeps; one
                                       power iteration or none may then do. Only for calls whose U
                                       holds such a result (not the first inversion) */
  KFAC_OPT_SPLIT_TARGET = 15,       /* [0 = 152]: a tensor-core product with fewer output tiles
                                       than 4/5 of this many CTAs and K >= 1024 splits K into
                                       chunks of at least 512 so that up to this many CTAs
                                       share it, summed by a reducing epilogue; -1 = never */
  KFAC_OPT_TAIL_PLANES = 19,        /* [1]: FP32 (3xTF32) products read precomputed TF32 tails
                                       of their large operands (the factor's once per
                                       inversion, 4 d^2 bytes of workspace per concurrent
                                       item; the batch's and the k x d bases' per product)
                                       instead of every CTA forming them in shared memory;
                                       0 = form them in the kernel (less workspace). Results
                                       are bitwise the same either way */
  KFAC_OPT_CHOL_BLOCKED = 20,       /* [1]: FP32 Cholesky factors of order above 236 (CholeskyQR
                                       Grams and the eigensolver's C + sI) are computed blocked:
                                       one-CTA factorisations of diagonal blocks of at most 236,
                                       triangular solves and tensor-core (3xTF32) rank updates
                                       between them; 0 = on one thread-block cluster
                                       (KFAC_OPT_CHOL_CLUSTER, KFAC_OPT_CHOL_PANEL). With 1 the
                                       CholeskyQR solves Q^T = L^-1 Y^T of order above 288 are
                                       blocked the same way (the off-diagonal work as
                                       tensor-core products) */
  KFAC_OPT_TRSM_INVERSE = 21,       /* [0]: 1 = the CholeskyQR solves Q^T = L^-1 Y^T (Alg. 3's
                                       QR step) form L^-1 once by solving the k x k identity,
                                       then Q^T as one FP32-accurate tensor-core product with
                                       the transposed basis (2 k^2 d flops on the tensor cores):
                                       faster on some GPUs, but the explicit inverse of a nearly
                                       singular factor (a numerically rank-deficient sketch of
                                       a steep spectrum) can overflow; 0 = block substitution
                                       on the SIMT pipes (shared-memory solve, blocked above
                                       order 288). The autotuner leaves it as set */
  KFAC_OPT_CHOL_PANEL = 18,         /* [16]: panel width of the multi-CTA Cholesky, 16 or 32
                                       (halved while its shared memory overflows); wider panels
                                       take half the cluster barriers and broadcasts */
  KFAC_OPT_CHOL_CLUSTER = 14,       /* [0 = automatic]: CTAs of the multi-CTA FP32/FP64
                                       Cholesky used where the one-CTA kernel's shared memory
                                       cannot hold the k x k Gram (k > 236), 1..16; raised to
                                       the fewest CTAs that hold their rows. Fewer CTAs take
                                       fewer cluster barriers and broadcasts per panel and
                                       leave SMs to the other factors of a grouped call */
  KFAC_OPT_INVERT_METHOD = 13,      /* [0]: 0 = SREVD (Alg. 3, SRE-KFAC): U = Q P from the
                                       eigendecomposition of C = Q^T F Q; 1 = RSVD (Alg. 2, as
                                       RS-KFAC's Alg. 4 uses it): U = V~, the leading right
                                       singular vectors of B = Q^T F, and D = its singular
                                       values (Sec. 2.3: V~ carries a much smaller projection
                                       error than SREVD's U). B^T is orthonormalised by the same
                                       shifted CholeskyQR (B^T = Q2 R2) and R2 = Q2^T B^T is
                                       factored by one-sided Jacobi, so B B^T is never formed.
                                       Both apply to kfac_rsvd_invert and its grouped form; the
                                       direct path (k >= d) is the same for both */
  KFAC_OPT_GROUP_STREAMS = 12,      /* [16]: streams a grouped call forks from the context
                                       stream, 1..32 (1 = every item in turn on the context
                                       stream). More streams overlap more of the items'
                                       latency-bound k x k steps; each stream has its own
                                       workspace slice. The device runs at most
                                       CUDA_DEVICE_MAX_CONNECTIONS streams side by side (an
                                       environment variable read when the process creates its
                                       CUDA context; 8 unless set, up to 32): set it to 32
                                       for more than 8 streams to overlap (the Python binding
                                       defaults it to 32 on import) */
  KFAC_OPT_WAIT_CYCLES = 11,        /* [4e9, ~2 s]: limit, in SM clock cycles, of every wait
                                       in which one role of a tensor-core kernel waits for
                                       another (loads for the issuer, the issuer for free
                                       stages, ...), 1..1e12. A wait that runs out raises
                                       KFAC_FLAG_TIMEOUT (kfac_get_status then returns
                                       KFAC_ERR_TIMEOUT); the kernel still waits for its own
                                       copies and tensor-core operations in flight (with the
                                       default limit), writes zeros for the products it could
                                       not finish and returns. Small values exist to exercise
                                       that path */
  KFAC_OPT_EIG_REFINE_FP64 = 10     /* 0 [default]: the eigen-refinement and basis-polish
                                       k x k products run in FP32 (FP64 carries the matrices
                                       between steps); their rounding, ~6e-8 of ||C||, is at
                                       the accuracy the FP32-accurate projection C carries.
                                       1: FP64 products (FP64 issues at ~1/64 of the FP32
                                       rate on this part) */
} kfac_option;

KFAC_API kfac_status kfac_set_option(kfac_ctx* ctx, kfac_option opt, double value);

/* Utility exposing the GEMM engine the entry points above are built on (used
 * to test it directly): D = alpha * A B^T + beta * D for row-major A (M x K,
 * lda), B (N x K, ldb) and D (M x N, ldd), device pointers. prec: FP32 (3xTF32
 * tensor-core products), TF32 or BF16 (operands rounded, FP32 accumulation).
 * The products run on the tcgen05 tensor cores; an operand whose base or row
 * stride is not 16-byte aligned (which TMA cannot read) is first copied into a
 * padded workspace. D must not overlap A or B. */
KFAC_API kfac_status kfac_gemm_nt(kfac_ctx* ctx, int M, int N, int K, const float* A, int lda, const float* B,
                                  int ldb, float alpha, float beta, float* D, int ldd, kfac_precision prec);

/* Per-stage device timing (CUDA events recorded on the context stream around
 * every kernel group; off by default). kfac_profile_enable(ctx, 1) starts
 * recording and clears the totals. kfac_profile_read() synchronises the stream,
 * and for i < min(max_stages, KFAC_NUM_STAGES) stores the stage name (static
 * string), the summed device milliseconds and the number of timed launches,
 * sets *n_stages to the number of stages written, and clears the totals. */
#define KFAC_NUM_STAGES 16
KFAC_API kfac_status kfac_profile_enable(kfac_ctx* ctx, int on);
KFAC_API kfac_status kfac_profile_read(kfac_ctx* ctx, const char** names, double* total_ms, int* launches,
                                       int max_stages, int* n_stages);
/* The recorded stage intervals as a timeline (call before kfac_profile_read,
 * which clears them): synchronises the context stream, sets *n_events to the
 * number of intervals recorded since kfac_profile_enable(ctx, 1) and, for the
 * first min(max_events, *n_events) of them in order of start time, stores the
 * stage index (into the names kfac_profile_read reports), the grouped-call item
 * index (-1 outside a grouped call) and the start and end in milliseconds
 * after recording began. Any output pointer may be NULL. Intervals of items on
 * forked streams overlap; the timeline shows how. KFAC_ERR_INVALID_ARG if
 * recording was never enabled. */
KFAC_API kfac_status kfac_profile_timeline(kfac_ctx* ctx, int max_events, int* stage, int* item, double* start_ms,
                                           double* end_ms, int* n_events);
/* Name of stage index `stage` (a static string), NULL if out of range. */
KFAC_API const char* kfac_stage_name(int stage);

/* Number of kernels this library has launched in the process so far (all
 * contexts). Used to count device work inside a timed region. */
KFAC_API uint64_t kfac_kernel_launch_count(void);

/* Number of large products (EA SYRK, sketch / power / projection, lift,
 * preconditioner apply, kfac_gemm_nt) that ran on the SIMT fallback kernel
 * instead of the tensor cores, in the process so far. Operands whose rows are
 * not 16-byte aligned are copied to a padded workspace first, so this stays 0
 * unless a product is degenerate or kfac_precondition_noalloc's transposed
 * operands are used. */
KFAC_API uint64_t kfac_simt_gemm_count(void);

/* Device-side counters of the context, read after synchronising its stream and
 * then cleared: out[0] = Jacobi sweeps performed, out[1] = Jacobi solves,
 * out[2] = Gram Cholesky factorisations, out[3] = extra Cholesky shift attempts.
 * n = number of entries of out (at most 4 are written). */
KFAC_API kfac_status kfac_stats_read(kfac_ctx* ctx, int64_t* out, int n);

#ifdef __cplusplus
}
#endif

#endif /* KFAC_H_ */
