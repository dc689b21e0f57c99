// C ABI of libkfac: context, workspace, argument checks and the orchestration
// of the kernels that make up each entry point.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include "common.cuh"
#include "gemm.cuh"

namespace {
enum Stage {
  ST_EA, ST_TRANSPOSE, ST_SKETCH, ST_GRAM, ST_CHOL, ST_TRSM, ST_PROJ, ST_EIG, ST_REFINE, ST_SELECT, ST_LIFT,
  ST_APPLY_T, ST_APPLY_M, ST_APPLY_T2, ST_APPLY_S, ST_POLISH, ST_COUNT
};
const char* const kStageNames[ST_COUNT] = {
    "ea_syrk", "omega_transpose", "sketch_gemm", "cholqr_gram", "cholqr_chol", "cholqr_trsm", "projection_gram",
    "eig_jacobi", "eig_refine", "eig_select", "lift_gemm", "apply_T", "apply_M", "apply_T2", "apply_S",
    "basis_polish"};
static_assert(ST_COUNT == KFAC_NUM_STAGES, "stage table");

// CUDA-event pairs recorded around each kernel group when profiling is on.
struct Profiler {
  bool on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[ST_COUNT];
  std::vector<int> item[ST_COUNT];  // grouped-call item of each interval (-1: not in a grouped call)
  size_t used[ST_COUNT] = {};
  cudaEvent_t base = nullptr;  // recorded on the context stream when recording starts
  ~Profiler() {
    for (auto& v : ev)
      for (auto& p : v) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
    if (base) cudaEventDestroy(base);
  }
};
}  // namespace

constexpr int kMaxSideStreams = 32;

struct kfac_ctx {
  Profiler prof;
  cudaStream_t side[kMaxSideStreams] = {};  // forked streams for grouped calls
  cudaEvent_t join_ev[kMaxSideStreams] = {};
  cudaEvent_t fork_ev = nullptr;
  std::vector<cudaEvent_t> item_ev;  // kfac_step_grouped: one per factor (its inversion done)
  int device = 0;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int* dflags = nullptr;  // device status word the kernels being enqueued raise flags in
  int* dglobal = nullptr;  // the context's own status word (dflags outside grouped calls)
  int* ditems = nullptr;   // per-item status words of grouped calls (item_cap of them)
  int item_cap = 0, item_used = 0;
  unsigned long long* dstats = nullptr;  // STAT_COUNT device counters
  // options
  int cholqr_passes = 3;
  int cholqr_inner_passes = 3;
  int cholqr_fp32_passes = 6;
  int basis_polish = 1;
  int cholqr_inner_fp32 = 1;
  double cholqr_shift = 1e-5;
  int eig_refine = 1;
  int eig_max_sweeps = 40;
  double eig_tol = 2e-6;
  double eig_stop_tol = 3e-3;
  int eig_refine_fp64 = 0;
  long long wait_cycles = kfac::kDefaultWaitCycles;
  int group_streams = 16;  // side streams a grouped call may fork (KFAC_OPT_GROUP_STREAMS)
  int invert_method = 0;   // KFAC_OPT_INVERT_METHOD: 0 SREVD (Alg. 3), 1 RSVD V~ (Alg. 2, RS-KFAC)
  int chol_cluster = 0;    // KFAC_OPT_CHOL_CLUSTER: CTAs of the multi-CTA Cholesky (0 = automatic)
  int chol_panel = 16;     // KFAC_OPT_CHOL_PANEL: its panel width (16 or 32)
  int split_target = 0;    // KFAC_OPT_SPLIT_TARGET: CTAs a split-K product may fill (0 = 152, -1 = no split)
  int warm_start = 0;      // KFAC_OPT_WARM_START: previous U seeds the sketch
  long long conv_chunk = 32LL << 20;  // KFAC_OPT_CONV_CHUNK: floats of one patch-matrix chunk
  int tail_planes = 1;                // KFAC_OPT_TAIL_PLANES: precomputed 3xTF32 tails of the large operands
  int chol_blocked = 1;               // KFAC_OPT_CHOL_BLOCKED: blocked FP32 Cholesky above the one-CTA limit
  int trsm_inverse = 0;               // KFAC_OPT_TRSM_INVERSE: CholeskyQR solves through L^-1 and one product
};

namespace {

using namespace kfac;

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Bump allocator over the context workspace (256-byte aligned slices).
struct Bump {
  size_t off = 0;
  template <typename T>
  size_t take(size_t count) {
    size_t o = (off + 255) & ~size_t(255);
    off = o + count * sizeof(T);
    return o;
  }
};

kfac_status ensure_ws(kfac_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return KFAC_OK;
  if (ctx->ws) {
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return KFAC_ERR_CUDA;
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  size_t want = std::max(bytes, size_t(1) << 20);
  if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
    cudaGetLastError();
    return KFAC_ERR_OOM;
  }
  ctx->ws_bytes = want;
  return KFAC_OK;
}

template <typename T>
T* at(kfac_ctx* ctx, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(ctx->ws) + off);
}

#define CK(expr)                                   \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return KFAC_ERR_CUDA;   \
  } while (0)

inline long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

// Records a start event now and an end event when the scope closes.
struct StageScope {
  kfac_ctx* c;
  int st;
  long long idx = -1;
  StageScope(kfac_ctx* ctx, int stage) : c(ctx), st(stage) {
    Profiler& p = c->prof;
    if (!p.on) return;
    if (p.used[st] == p.ev[st].size()) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess) return;
      if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
      p.ev[st].push_back({a, b});
      p.item[st].push_back(-1);
    }
    idx = (long long)p.used[st]++;
    p.item[st][idx] = c->dflags == c->dglobal ? -1 : (int)(c->dflags - c->ditems);
    cudaEventRecord(p.ev[st][idx].first, c->stream);
  }
  ~StageScope() {
    if (idx >= 0) cudaEventRecord(c->prof.ev[st][idx].second, c->stream);
  }
};
#define STAGE(ctx, st) StageScope stage_scope_##st(ctx, st)

// ---- invert ------------------------------------------------------------------

struct InvertLayout {
  size_t om, y, q, part, g, g32, l32, gd, dinv, c, c32, x, lam, work, jac, r32, pt, qn, fp, fb, xb, skws, flo, xlo,
      xlo2, cb, tb, ti, total;
  long long dp, kp, dpb, skws_floats;
  int nsplit, kchunk;
  bool pack_f, bf16, tails;
};

constexpr int kSketchMaxSplit = 6;  // split-K partials of the sketch products

// pack_f: F's rows are not 16-byte aligned, so the sketch products read a
// copy of F with a padded row stride (one extra pass over F per inversion,
// against the q + 2 passes of the products it puts on the tensor cores).
// bf16: the BF16 products read a BF16 copy of F (made once per inversion) and
// of each product's k x d operand, which TMA feeds to the tensor cores as is.
// tails: the FP32 (3xTF32) products read precomputed tails of their operands
// (F's once per inversion, 4 d^2 bytes; the k x d operands' per product)
// instead of every CTA forming them in shared memory.
InvertLayout invert_layout(int d, int k, int r, bool pack_f, bool bf16 = false, bool tails = false) {
  InvertLayout L = {};
  Bump b;
  L.pack_f = pack_f;
  L.bf16 = bf16 && k < d;
  L.tails = tails && !L.bf16 && k < d;
  if (k >= d) {  // exact path
    int n = d;
    L.c = b.take<double>((size_t)n * n);
    L.x = b.take<double>((size_t)n * n);
    L.lam = b.take<double>(n);
    L.work = b.take<double>(eig_refine_doubles(n));
    L.jac = b.take<float>(eig_scratch_floats(n));
    L.r32 = b.take<float>(eig_refine_floats(n));
    L.total = b.off;
    return L;
  }
  L.dp = round_up(d, 4);
  // Grams (k x k, K = d): symmetric ones are computed on the upper tiles only
  // (t (t + 1) / 2 of 128 x 128, t = ceil(k / 128)); K is split so that about
  // one CTA per SM works on a Gram, each over at least 256 of K (a CTA's
  // pipeline fill and epilogue then stay small against its main loop).
  {
    const long long t = (k + 127) / 128, tiles = t * (t + 1) / 2;
    const long long cap = std::max<long long>(1, std::min<long long>(32, d / 256));
    L.nsplit = (int)std::min<long long>(cap, std::max<long long>(1, (152 + tiles / 2) / tiles));
  }
  L.kchunk = (int)round_up((d + L.nsplit - 1) / L.nsplit, 64);
  L.nsplit = (d + L.kchunk - 1) / L.kchunk;
  L.om = b.take<float>((size_t)k * L.dp);
  L.y = b.take<float>((size_t)k * L.dp);
  L.q = b.take<float>((size_t)k * L.dp);
  L.part = b.take<float>((size_t)L.nsplit * k * k);
  L.g = b.take<double>((size_t)k * k);
  L.g32 = b.take<float>((size_t)k * k);
  L.l32 = b.take<float>((size_t)k * k);
  L.gd = b.take<double>((size_t)k);
  L.cb = b.take<char>(chol_blocked_ws_bytes(k));
  L.tb = b.take<char>(trsm_blocked_ws_bytes(k, d));
  L.ti = b.take<char>(trsm_inverse_ws_bytes(k, d));
  L.dinv = b.take<float>(trsm_ws_floats(k));
  L.c = b.take<double>((size_t)k * k);
  L.c32 = b.take<float>((size_t)k * k);
  L.x = b.take<double>((size_t)k * k);
  L.lam = b.take<double>(k);
  L.work = b.take<double>(eig_refine_doubles(k));
  L.jac = b.take<float>(eig_scratch_floats(k));
  L.r32 = b.take<float>(eig_refine_floats(k) + polish_floats(k));  // refinement, then the polish's E, P, Q
  L.kp = round_up(k, 4);
  L.pt = b.take<float>((size_t)r * L.kp);  // P[:, :r]^T, the lift's B operand
  L.qn = b.take<float>((size_t)d * L.kp);  // Q (d x k), the lift's A operand
  if (pack_f) L.fp = b.take<float>((size_t)d * L.dp);
  L.dpb = round_up(d, 8);
  if (L.bf16) {
    L.fb = b.take<uint16_t>((size_t)d * L.dpb);
    L.xb = b.take<uint16_t>((size_t)k * L.dpb);
  }
  L.skws_floats = (long long)kSketchMaxSplit * k * d;
  L.skws = b.take<float>((size_t)L.skws_floats);
  if (L.tails) {
    L.flo = b.take<float>((size_t)d * L.dp);
    L.xlo = b.take<float>((size_t)k * L.dp);
    L.xlo2 = b.take<float>((size_t)k * L.dp);
  }
  L.total = b.off;
  return L;
}

// Gram-type product out = A A'^T (k x k, K = d) for two k x d row-major
// operands, split over K with FP32 partials summed with compensation (and
// symmetrised) into FP64.
// a_tails_ready: L.xlo already holds A's TF32 tails (stored by the solve that produced A).
kfac_status gram_f64(kfac_ctx* ctx, const InvertLayout& L, const float* A, const float* Bm, long long ld, int k,
                     int d, kfac_precision prec, double* out, int stage, float* out32, int symmetrize = 1,
                     double* dscale = nullptr, bool a_tails_ready = false) {
  GemmDesc<float> g = {};
  g.M = k; g.N = k; g.K = d;
  g.A = A; g.sam = ld; g.sak = 1;
  g.B = Bm; g.sbn = ld; g.sbk = 1;
  g.D = at<float>(ctx, L.part); g.ldd = k;
  g.alpha = 1.0f;
  g.zsplit = L.nsplit; g.kchunk = L.kchunk; g.zstride = (long long)k * k;
  // A A^T: only the tiles at and above the diagonal, the reduce mirrors them
  const bool upper = A == Bm && symmetrize == 1;
  g.sym = upper ? 1 : 0;
  g.flags = ctx->dflags; g.wait_cycles = ctx->wait_cycles; g.split_target = ctx->split_target;
  StageScope sc(ctx, stage);
  if (L.tails && prec == KFAC_PREC_FP32) {
    if (!a_tails_ready) CK(tails_f32(A, ld, k, d, at<float>(ctx, L.xlo), L.dp, ctx->stream));
    g.A_lo = at<float>(ctx, L.xlo); g.ld_alo = L.dp;
    if (Bm != A) CK(tails_f32(Bm, ld, k, d, at<float>(ctx, L.xlo2), L.dp, ctx->stream));
    g.B_lo = at<float>(ctx, Bm != A ? L.xlo2 : L.xlo); g.ld_blo = L.dp;
  }
  CK(gemm_f32(g, prec, ctx->stream));
  CK(reduce_splitk_f64(at<float>(ctx, L.part), L.nsplit, g.zstride, k, k, out, k, upper ? 2 : symmetrize,
                       ctx->dflags, ctx->stream, out32, dscale));
  return KFAC_OK;
}

// Yt_out (k x d) = Xt (k x d) F: the sketch / power / projection product,
// computed as (F Xt^T)^T. F is the large operand (A, M = d rows streamed once),
// Xt the small one (B, N = k); the transposed store of the d x k product lands
// row-major in Yt. F is symmetric, so A(m, kk) = F[m][kk] reads F row-major.
kfac_status sketch_product(kfac_ctx* ctx, const InvertLayout& L, const float* Xt, long long ldx, const float* F,
                           int ldf, int k, int d, kfac_precision prec, float* out, long long ldo,
                           bool x_tails_ready = false) {
  GemmDesc<float> g = {};
  g.M = d; g.N = k; g.K = d;
  g.A = F; g.sam = ldf; g.sak = 1;
  g.B = Xt; g.sbn = ldx; g.sbk = 1;
  if (L.bf16 && prec == KFAC_PREC_BF16) {  // BF16 copies: F's made once per inversion, Xt's here
    STAGE(ctx, ST_TRANSPOSE);
    CK(to_bf16_f32(Xt, ldx, k, d, at<uint16_t>(ctx, L.xb), L.dpb, ctx->stream));
    g.A = reinterpret_cast<const float*>(at<uint16_t>(ctx, L.fb)); g.sam = L.dpb;
    g.B = reinterpret_cast<const float*>(at<uint16_t>(ctx, L.xb)); g.sbn = L.dpb;
    g.ab_bf16 = 1;
  }
  g.D = out; g.ldd = ldo; g.d_trans = 1;
  g.alpha = 1.0f; g.zsplit = 1;
  g.ws = at<float>(ctx, L.skws); g.ws_floats = L.skws_floats;
  g.flags = ctx->dflags; g.wait_cycles = ctx->wait_cycles; g.split_target = ctx->split_target;
  STAGE(ctx, ST_SKETCH);
  if (L.tails && prec == KFAC_PREC_FP32) {  // F's tails were formed once per inversion
    if (!x_tails_ready) CK(tails_f32(Xt, ldx, k, d, at<float>(ctx, L.xlo), L.dp, ctx->stream));
    g.A_lo = at<float>(ctx, L.flo); g.ld_alo = L.dp;
    g.B_lo = at<float>(ctx, L.xlo); g.ld_blo = L.dp;
  }
  CK(gemm_f32(g, prec, ctx->stream));
  return KFAC_OK;
}

// `final_basis`: the basis the eigenpairs are taken in (the last one of Alg. 3);
// a basis that only feeds the next power iteration may factor every pass in
// FP32 (KFAC_OPT_CHOLQR_INNER_FP32).
// *tails_ready (optional): on return, whether L.xlo holds the TF32 tails of the
// basis in cur (the shared-memory substitution solve stores them beside it).
kfac_status orthonormalise(kfac_ctx* ctx, const InvertLayout& L, float*& cur, float*& other, int k, int d,
                           int passes, bool final_basis, bool* tails_ready = nullptr) {
  bool ready = false;  // L.xlo holds the tails of cur
  for (int pass = 0; pass < passes; ++pass) {
    // Passes after the first factor the column-scaled Gram D^-1 G D^-1 (unit
    // diagonal, D = diag(G)^1/2) and solve with D chol(D^-1 G D^-1 + s I): a
    // column that the shifted pass before left far below unit length (the
    // directions of a numerically rank-deficient sketch) is normalised instead
    // of staying short, and the shifts and the pivot floor act relative to
    // each column's own length.
    double* dscale = pass > 0 ? at<double>(ctx, L.gd) : nullptr;
    kfac_status st = gram_f64(ctx, L, cur, cur, L.dp, k, d, KFAC_PREC_FP32, at<double>(ctx, L.g), ST_GRAM,
                              at<float>(ctx, L.g32), 1, dscale, ready);
    if (st != KFAC_OK) return st;
    {
      STAGE(ctx, ST_CHOL);
      // First pass: shift relative to trace(G) (the sketch may be ill-conditioned
      // beyond the FP32 Gram's accuracy). Middle passes: a shift of 1e-5 of the
      // mean diagonal, above the FP32-accurate Gram's rounding noise (~1e-6 of
      // it), so the directions the first pass left at noise level cannot make
      // the factorisation indefinite; the last pass (a near-orthonormal basis)
      // is unshifted.
      const double shift = pass == 0 ? ctx->cholqr_shift : (pass + 1 < passes ? -1e-5 : 0.0);
      const bool fp64 = (final_basis || !ctx->cholqr_inner_fp32) &&
                        (pass >= ctx->cholqr_fp32_passes || (pass + 1 == passes && ctx->cholqr_fp32_passes < passes));
      if (!fp64 && ctx->chol_blocked && chol_blocked_ws_bytes(k) > 0)
        CK(chol_blocked(at<double>(ctx, L.g), at<float>(ctx, L.g32), k, k, shift, at<float>(ctx, L.l32), ctx->dflags,
                        ctx->dstats, ctx->stream, nullptr, at<char>(ctx, L.cb), ctx->wait_cycles));
      else
        CK(chol_cluster(at<double>(ctx, L.g), k, shift, fp64, at<float>(ctx, L.l32), ctx->dflags, ctx->dstats,
                        ctx->stream, nullptr, at<float>(ctx, L.g32), k, ctx->chol_cluster, ctx->chol_panel));
      if (dscale && !ctx->trsm_inverse) CK(factor_unscale(at<float>(ctx, L.l32), k, dscale, ctx->stream));
    }
    ready = false;
    {
      STAGE(ctx, ST_TRSM);
      if (ctx->trsm_inverse) {
        CK(trsm_inverse(at<float>(ctx, L.l32), k, cur, L.dp, other, L.dp, d, at<char>(ctx, L.ti), ctx->dflags,
                        ctx->wait_cycles, ctx->stream, dscale));
      } else if (ctx->chol_blocked && trsm_blocked_used(k)) {
        CK(trsm_blocked(at<float>(ctx, L.l32), k, cur, L.dp, other, L.dp, d, at<char>(ctx, L.tb), ctx->dflags,
                        ctx->wait_cycles, ctx->stream));
      } else {  // the solve stores the new basis's tails beside it: no tails pass before its next product
        float* qlo = L.tails ? at<float>(ctx, L.xlo) : nullptr;
        CK(trsm_lower_f32(at<float>(ctx, L.l32), k, cur, L.dp, other, L.dp, d, at<float>(ctx, L.dinv), ctx->stream,
                          qlo, L.dp));
        ready = qlo != nullptr;
      }
    }
    std::swap(cur, other);
  }
  if (tails_ready) *tails_ready = ready;
  return KFAC_OK;
}

kfac_status eigensolve(kfac_ctx* ctx, const double* C, const float* C32, long long ld32, int n, double* X,
                       double* lam, double* work, float* jac, float* r32) {
  {
    STAGE(ctx, ST_EIG);
    CK(eig_jacobi_f32(C, n, 1e-6, ctx->eig_max_sweeps, (float)ctx->eig_tol, (float)ctx->eig_stop_tol, X, lam, jac,
                      ctx->dflags, ctx->dstats, ctx->stream, C32, ld32, ctx->chol_cluster, ctx->chol_panel,
                      ctx->chol_blocked, ctx->wait_cycles));
  }
  STAGE(ctx, ST_REFINE);
  for (int it = 0; it < ctx->eig_refine; ++it) {
    if (ctx->eig_refine_fp64) CK(eig_refine_f64(C, n, X, lam, work, ctx->dflags, ctx->stream));
    else CK(eig_refine_f32(C32, ld32, n, X, lam, r32, work, ctx->dflags, ctx->stream));
  }
  return KFAC_OK;
}


// D = A B for k x k row-major FP64 matrices.
cudaError_t small_product_f64(const double* A, const double* B, double* D, int k, cudaStream_t s) {
  GemmDesc<double> g = {};
  g.M = k; g.N = k; g.K = k; g.alpha = 1.0; g.beta = 0.0; g.zsplit = 1;
  g.A = A; g.sam = k; g.sak = 1;
  g.B = B; g.sbn = 1; g.sbk = k;  // B(n, kk) = B[kk][n]
  g.D = D; g.ldd = k;
  return gemm_simt_f64(g, s);
}

kfac_status check_invert(const kfac_invert_desc& a, int* r_out, int* k_out) {
  if (a.d <= 0 || !a.F || a.ldf < a.d || a.rank <= 0 || a.oversample < 0 || a.power_iters < 0 || a.power_iters > 64)
    return KFAC_ERR_INVALID_ARG;
  if (!(a.lambda > 0.0f) || a.prec < KFAC_PREC_FP32 || a.prec > KFAC_PREC_BF16) return KFAC_ERR_INVALID_ARG;
  const int r = std::min(a.rank, a.d);
  const long long kl = (long long)a.rank + a.oversample;
  if (!a.U || a.ldu < r || !a.D || !a.coef) return KFAC_ERR_INVALID_ARG;
  const bool exact = kl >= a.d;
  if (!exact && a.omega && a.ldo < kl) return KFAC_ERR_INVALID_ARG;  // NULL omega: drawn from a.seed
  if ((exact ? (long long)a.d : kl) > kMaxSketch) return KFAC_ERR_UNSUPPORTED;
  const int k = (int)kl;
  *r_out = r;
  *k_out = k;
  return KFAC_OK;
}

// Lift U (d x r) = Qb P[:, :r] from the basis Qb^T (k x d, row stride L.dp) and
// P[:, :r]^T in L.pt: Qb transposed into L.qn, then a tcgen05 product with both
// operands K-contiguous.
kfac_status lift(kfac_ctx* ctx, const InvertLayout& L, const float* Qbt, const kfac_invert_desc& a, int d, int k,
                 int r) {
  STAGE(ctx, ST_LIFT);
  float* Qn = at<float>(ctx, L.qn);
  CK(transpose_f32(Qbt, L.dp, k, d, Qn, L.kp, ctx->stream));
  GemmDesc<float> g = {};
  g.M = d; g.N = r; g.K = k;
  g.A = Qn; g.sam = L.kp; g.sak = 1;
  g.B = at<float>(ctx, L.pt); g.sbn = L.kp; g.sbk = 1;
  g.D = a.U; g.ldd = a.ldu;
  g.alpha = 1.0f; g.zsplit = 1;
  g.flags = ctx->dflags; g.wait_cycles = ctx->wait_cycles; g.split_target = ctx->split_target;
  CK(gemm_f32(g, KFAC_PREC_FP32, ctx->stream));
  return KFAC_OK;
}

// RS-KFAC's inverse factors (Alg. 2 with the power iterations of Sec. 2.2, as
// Alg. 4 uses them), from the final basis Q^T (in cur): B = Q^T F (k x d, held
// as B^T's columns in the rows of Z^T); B^T = Q2 R2 by the same shifted
// CholeskyQR (Q2 orthonormal, d x k); R2 = Q2^T B^T (k x k, FP32-accurate
// product kept in FP64); the SVD R2 = U_R diag(s) W^T by one-sided Jacobi, so
// B^T = (Q2 U_R) diag(s) W^T and the right singular vectors of B are
// V_B = Q2 U_R. Outputs V~ = (Q2 U_R)[:, :r] in U, D = s[:r] and the Eq. (13)
// coefficients from s. The SVD of the triangular-like R2 never forms B B^T,
// so the singular values keep an absolute error ~u s_1 (not u s_1^2 / s_i).
kfac_status rsvd_tail(kfac_ctx* ctx, const kfac_invert_desc& a, const InvertLayout& L, float* cur, float* other, int d,
                      int k, int r, const float* F, int ldf) {
  cudaStream_t s = ctx->stream;
  kfac_status st = sketch_product(ctx, L, cur, L.dp, F, ldf, k, d, a.prec, other, L.dp);  // Z^T = Q^T F = B
  if (st != KFAC_OK) return st;
  float* c1 = at<float>(ctx, L.om);  // Omega^T is dead: B^T's basis is built there and in cur
  CK(cudaMemcpyAsync(c1, other, sizeof(float) * (size_t)k * L.dp, cudaMemcpyDeviceToDevice, s));
  st = orthonormalise(ctx, L, c1, cur, k, d, ctx->cholqr_passes, true);  // Q2^T in c1
  if (st != KFAC_OK) return st;
  st = gram_f64(ctx, L, c1, other, L.dp, k, d, KFAC_PREC_FP32, at<double>(ctx, L.c), ST_PROJ, at<float>(ctx, L.c32),
                0);  // R2 = Q2^T B^T, not symmetric
  if (st != KFAC_OK) return st;
  // Newton-Schulz polish of Q2 (as for SREVD's basis): with E = Q2^T Q2 - I and
  // M = I - E/2, Q2 M is orthonormal to second order and B^T = (Q2 M)(M R2) to
  // first order, so the SVD is taken of M R2 and V~ = Q2 (M U_R).
  float* pw32 = at<float>(ctx, L.r32) + eig_refine_floats(k);
  const bool polish = ctx->basis_polish != 0;
  if (polish) {
    st = gram_f64(ctx, L, c1, c1, L.dp, k, d, KFAC_PREC_FP32, at<double>(ctx, L.g), ST_POLISH, nullptr);
    if (st != KFAC_OK) return st;
    STAGE(ctx, ST_POLISH);
    CK(polish_E_f32(at<double>(ctx, L.g), k, pw32, s));
    CK(polish_vectors_f32(at<double>(ctx, L.c), k, pw32, s));  // R2 <- M R2
    CK(convert_f64_to_f32(at<double>(ctx, L.c), (long long)k * k, at<float>(ctx, L.c32), s));
  }
  {
    STAGE(ctx, ST_EIG);
    // Swept to full convergence (every pair cosine <= KFAC_OPT_EIG_TOL): no
    // refinement step follows here to square away an early stop's residue.
    CK(svd_jacobi_f32(at<float>(ctx, L.c32), k, ctx->eig_max_sweeps, (float)ctx->eig_tol, 0.0f, at<double>(ctx, L.x),
                      at<double>(ctx, L.lam), at<float>(ctx, L.jac), ctx->dflags, ctx->dstats, s));
  }
  if (polish) {
    STAGE(ctx, ST_POLISH);
    CK(polish_vectors_f32(at<double>(ctx, L.x), k, pw32, s));  // U_R <- M U_R
  }
  {
    STAGE(ctx, ST_SELECT);
    CK(eig_select(at<double>(ctx, L.x), at<double>(ctx, L.lam), k, r, a.lambda, at<float>(ctx, L.pt), L.kp, a.D,
                  a.coef, nullptr, 0, s, /*singular=*/1));
  }
  return lift(ctx, L, c1, a, d, k, r);
}

// The randomized inversion of one factor, enqueued on ctx->stream, with its
// workspace slices offset by `base` bytes.
kfac_status invert_run(kfac_ctx* ctx, const kfac_invert_desc& a, InvertLayout L, size_t base) {
  const int d = a.d, r = std::min(a.rank, a.d), k = a.rank + a.oversample;
  const float* F = a.F;
  int ldf = a.ldf;
  for (size_t* o : {&L.om, &L.y, &L.q, &L.part, &L.g, &L.g32, &L.l32, &L.gd, &L.dinv, &L.c, &L.c32, &L.x, &L.lam, &L.work,
                    &L.jac, &L.r32, &L.pt, &L.qn, &L.fp, &L.fb, &L.xb, &L.skws, &L.flo, &L.xlo, &L.xlo2, &L.cb, &L.tb,
                    &L.ti})
    *o += base;
  cudaStream_t s = ctx->stream;
  kfac_status st;
  if (k >= d) {  // nothing to sketch: diagonalise F itself (Q = I)
    double* C = at<double>(ctx, L.c);
    CK(convert_f32_to_f64(F, ldf, d, d, C, d, ctx->dflags, s));
    st = eigensolve(ctx, C, F, ldf, d, at<double>(ctx, L.x), at<double>(ctx, L.lam), at<double>(ctx, L.work),
                    at<float>(ctx, L.jac), at<float>(ctx, L.r32));
    if (st != KFAC_OK) return st;
    STAGE(ctx, ST_SELECT);
    CK(eig_select(at<double>(ctx, L.x), at<double>(ctx, L.lam), d, r, a.lambda, nullptr, 0, a.D, a.coef, a.U,
                  a.ldu, s));
    return KFAC_OK;
  }
  if (L.pack_f) {  // rows of F not 16-byte aligned: the tensor-core products read a padded copy
    STAGE(ctx, ST_TRANSPOSE);
    float* Fp = at<float>(ctx, L.fp);
    CK(pack_rows_f32(F, ldf, d, d, Fp, L.dp, s));
    F = Fp;
    ldf = (int)L.dp;
  }
  if (L.bf16) {  // F rounded to BF16 once, for the sketch, power and projection products
    STAGE(ctx, ST_TRANSPOSE);
    CK(to_bf16_f32(F, ldf, d, d, at<uint16_t>(ctx, L.fb), L.dpb, s));
  }
  if (L.tails && a.prec == KFAC_PREC_FP32) {  // F's 3xTF32 tails once, for the sketch, power and projection products
    STAGE(ctx, ST_TRANSPOSE);
    CK(tails_f32(F, ldf, d, d, at<float>(ctx, L.flo), L.dp, s));
  }
  // Omega^T (k x d) so that every sketch product reads K-contiguous rows.
  float* Om = at<float>(ctx, L.om);
  float* cur = at<float>(ctx, L.y);
  float* other = at<float>(ctx, L.q);
  {
    STAGE(ctx, ST_TRANSPOSE);
    // Subspace iteration across inversions (warm start): the previous
    // inversion's U (the caller's U buffer, read before this call overwrites
    // it) seeds the first r sketch columns, omega's first k - r columns the rest.
    const int r0 = ctx->warm_start ? r : 0;
    if (r0 > 0) CK(transpose_f32(a.U, a.ldu, d, r, Om, L.dp, s));
    if (a.omega) CK(transpose_f32(a.omega, a.ldo, d, k - r0, Om + (size_t)r0 * L.dp, L.dp, s));
    else CK(draw_omega_f32(d, k, a.seed, 0, k - r0, Om + (size_t)r0 * L.dp, L.dp, true, s));
  }
  st = sketch_product(ctx, L, Om, L.dp, F, ldf, k, d, a.prec, cur, L.dp);  // Y^T = Omega^T F
  if (st != KFAC_OK) return st;
  for (int it = 0;; ++it) {
    bool q_tails = false;
    st = orthonormalise(ctx, L, cur, other, k, d,
                        it == a.power_iters ? ctx->cholqr_passes : ctx->cholqr_inner_passes,
                        it == a.power_iters, &q_tails);  // Q^T in cur
    if (st != KFAC_OK) return st;
    if (it == a.power_iters) break;
    st = sketch_product(ctx, L, cur, L.dp, F, ldf, k, d, a.prec, other, L.dp, q_tails);  // Y^T = Q^T F
    if (st != KFAC_OK) return st;
    std::swap(cur, other);
  }
  if (ctx->invert_method == 1) return rsvd_tail(ctx, a, L, cur, other, d, k, r, F, ldf);
  // Newton-Schulz polish of the final basis, in the k x k space: M = (3I - Q^T Q)/2
  // makes Q M orthonormal to second order; the Rayleigh-Ritz step below uses
  // Q M (C <- M C M, X <- M X) without touching the d x k basis.
  // With FP32 products (default) the polish works on E = Q^T Q - I (M = I - E/2);
  // the FP64 form builds M and multiplies by it.
  const bool polish = ctx->basis_polish != 0, polish64 = polish && ctx->eig_refine_fp64;
  float* pw32 = at<float>(ctx, L.r32) + eig_refine_floats(k);  // E, P, Q of the FP32 polish
  double* Mpol = nullptr;
  if (polish) {
    st = gram_f64(ctx, L, cur, cur, L.dp, k, d, KFAC_PREC_FP32, at<double>(ctx, L.g), ST_POLISH, nullptr);
    if (st != KFAC_OK) return st;
    if (polish64) {
      STAGE(ctx, ST_POLISH);
      CK(polish_factor(at<double>(ctx, L.g), k, s));
      Mpol = at<double>(ctx, L.g);
    }
  }
  // Projection C = Q^T F Q = Q^T (F Q): Z^T = Q^T F into `other`, then C = Q^T Z.
  st = sketch_product(ctx, L, cur, L.dp, F, ldf, k, d, a.prec, other, L.dp);
  if (st != KFAC_OK) return st;
  double* C = at<double>(ctx, L.c);
  st = gram_f64(ctx, L, cur, other, L.dp, k, d, KFAC_PREC_FP32, C, ST_PROJ, at<float>(ctx, L.c32));
  if (st != KFAC_OK) return st;
  if (Mpol) {  // C <- M (C M), with its FP32 copy for the eigensolver's factorisation
    STAGE(ctx, ST_POLISH);
    double* T = at<double>(ctx, L.work);
    CK(small_product_f64(C, Mpol, T, k, s));
    CK(small_product_f64(Mpol, T, C, k, s));
    CK(convert_f64_to_f32(C, (long long)k * k, at<float>(ctx, L.c32), s));
  } else if (polish) {
    STAGE(ctx, ST_POLISH);
    CK(polish_projected_f32(at<double>(ctx, L.g), C, at<float>(ctx, L.c32), k, pw32, s));
  }
  st = eigensolve(ctx, C, at<float>(ctx, L.c32), k, k, at<double>(ctx, L.x), at<double>(ctx, L.lam),
                  at<double>(ctx, L.work), at<float>(ctx, L.jac), at<float>(ctx, L.r32));
  if (st != KFAC_OK) return st;
  if (Mpol) {  // eigenvectors in the polished basis: X <- M X
    STAGE(ctx, ST_POLISH);
    double* T = at<double>(ctx, L.work);
    CK(small_product_f64(Mpol, at<double>(ctx, L.x), T, k, s));
    CK(cudaMemcpyAsync(at<double>(ctx, L.x), T, sizeof(double) * (size_t)k * k, cudaMemcpyDeviceToDevice, s));
  } else if (polish) {
    STAGE(ctx, ST_POLISH);
    CK(polish_vectors_f32(at<double>(ctx, L.x), k, pw32, s));
  }
  {
    STAGE(ctx, ST_SELECT);
    CK(eig_select(at<double>(ctx, L.x), at<double>(ctx, L.lam), k, r, a.lambda, at<float>(ctx, L.pt), L.kp, a.D,
                  a.coef, nullptr, 0, s));
  }
  // Lift: U (d x r) = Q P[:, :r], both operands K-contiguous (Q from Q^T by a
  // transpose, P[:, :r]^T from the selection) so the product runs on tcgen05.
  return lift(ctx, L, cur, a, d, k, r);
}


// Workspace of one preconditioner apply. All products read K-contiguous
// operands: T = J U_a diag(c_a) (d_g x r_a), M^T = U_a T^T + J^T/lam (d_a x d_g),
// T2^T = M^T U_g diag(c_g) (d_a x r_g), S = U_g (T2^T)^T + M/lam, with the small
// transposes U_a^T, U_g^T; split-K partials for the two long-K products.
struct PrecLayout {
  size_t uat, ugt, t, mt, t2, ws, jp, uap, ugp, big_lo, ua_lo, ug_lo, uat_lo, ugt_lo, t_lo, t2_lo, total;
  long long ld_uat, ld_ugt, ld_t, ld_mt, ld_t2, ws_floats, ld_jp, ld_uap, ld_ugp;
  bool pack_j, pack_ua, pack_ug, tails;
};

constexpr int kApplyMaxSplit = 6;

// pack_j / pack_ua / pack_ug: that operand's rows are not 16-byte aligned, so
// the tensor-core products read a copy with a padded row stride. tails: the
// FP32 products read precomputed 3xTF32 tails of their operands (one d_g x d_a
// plane serves J's and then M^T's).
PrecLayout prec_layout(int dg, int da, int ra, int rg, bool pack_j, bool pack_ua, bool pack_ug, bool tails = false) {
  PrecLayout P = {};
  Bump b;
  P.pack_j = pack_j; P.pack_ua = pack_ua && ra > 0; P.pack_ug = pack_ug && rg > 0;
  P.tails = tails;
  P.ld_uat = round_up(da, 4);
  P.ld_ugt = round_up(dg, 4);
  P.ld_t = round_up(std::max(ra, 1), 4);
  P.ld_mt = round_up(dg, 4);
  P.ld_t2 = round_up(std::max(rg, 1), 4);
  P.uat = b.take<float>((size_t)std::max(ra, 1) * P.ld_uat);
  P.ugt = b.take<float>((size_t)std::max(rg, 1) * P.ld_ugt);
  P.t = b.take<float>((size_t)dg * P.ld_t);
  P.mt = b.take<float>((size_t)da * P.ld_mt);
  P.t2 = b.take<float>((size_t)da * P.ld_t2);
  P.ws_floats = (long long)kApplyMaxSplit * std::max((long long)dg * std::max(ra, 1), (long long)da * std::max(rg, 1));
  P.ws = b.take<float>((size_t)P.ws_floats);
  P.ld_jp = round_up(da, 4);
  P.ld_uap = round_up(std::max(ra, 1), 4);
  P.ld_ugp = round_up(std::max(rg, 1), 4);
  if (P.pack_j) P.jp = b.take<float>((size_t)dg * P.ld_jp);
  if (P.pack_ua) P.uap = b.take<float>((size_t)da * P.ld_uap);
  if (P.pack_ug) P.ugp = b.take<float>((size_t)dg * P.ld_ugp);
  if (P.tails) {
    P.big_lo = b.take<float>(std::max((size_t)dg * P.ld_jp, (size_t)da * P.ld_mt));
    P.ua_lo = b.take<float>((size_t)da * P.ld_uap);
    P.ug_lo = b.take<float>((size_t)dg * P.ld_ugp);
    P.uat_lo = b.take<float>((size_t)std::max(ra, 1) * P.ld_uat);
    P.ugt_lo = b.take<float>((size_t)std::max(rg, 1) * P.ld_ugt);
    P.t_lo = b.take<float>((size_t)dg * P.ld_t);
    P.t2_lo = b.take<float>((size_t)da * P.ld_t2);
  }
  P.total = b.off;
  return P;
}

PrecLayout prec_layout_for(int dg, int da, const float* J, int ldj, const float* U_a, int ld_ua, int ra,
                           const float* U_g, int ld_ug, int rg, bool tails) {
  return prec_layout(dg, da, ra, rg, !tma_rows_ok(J, ldj), !tma_rows_ok(U_a, ld_ua), !tma_rows_ok(U_g, ld_ug), tails);
}

kfac_status precondition_run(kfac_ctx* ctx, int d_g, int d_a, const float* J, int ldj, const float* U_a, int ld_ua,
                             const float* coef_a, int r_a, const float* U_g, int ld_ug, const float* coef_g, int r_g,
                             float lambda, kfac_precision prec, float* S, int lds, PrecLayout P, size_t base) {
  for (size_t* o : {&P.uat, &P.ugt, &P.t, &P.mt, &P.t2, &P.ws, &P.jp, &P.uap, &P.ugp, &P.big_lo, &P.ua_lo, &P.ug_lo,
                    &P.uat_lo, &P.ugt_lo, &P.t_lo, &P.t2_lo})
    *o += base;
  cudaStream_t s = ctx->stream;
  const float inv_lam = 1.0f / lambda;
  const bool tails = P.tails && prec == KFAC_PREC_FP32;
  // Tails of a product's operand, formed just before the product reads it.
  auto tail = [&](GemmDesc<float>& g, bool a_side, const float* X, long long ldx, int rows, int cols, size_t plane,
                  long long ldp) -> cudaError_t {
    if (!tails || rows <= 0 || cols <= 0) return cudaSuccess;
    float* lo = at<float>(ctx, plane);
    cudaError_t e = tails_f32(X, ldx, rows, cols, lo, ldp, s);
    if (a_side) { g.A_lo = lo; g.ld_alo = ldp; } else { g.B_lo = lo; g.ld_blo = ldp; }
    return e;
  };
  if (P.pack_j || P.pack_ua || P.pack_ug) {  // operands whose rows TMA cannot read: padded copies
    STAGE(ctx, ST_TRANSPOSE);
    if (P.pack_j) {
      CK(pack_rows_f32(J, ldj, d_g, d_a, at<float>(ctx, P.jp), P.ld_jp, s));
      J = at<float>(ctx, P.jp);
      ldj = (int)P.ld_jp;
    }
    if (P.pack_ua) {
      CK(pack_rows_f32(U_a, ld_ua, d_a, r_a, at<float>(ctx, P.uap), P.ld_uap, s));
      U_a = at<float>(ctx, P.uap);
      ld_ua = (int)P.ld_uap;
    }
    if (P.pack_ug) {
      CK(pack_rows_f32(U_g, ld_ug, d_g, r_g, at<float>(ctx, P.ugp), P.ld_ugp, s));
      U_g = at<float>(ctx, P.ugp);
      ld_ug = (int)P.ld_ugp;
    }
  }
  float* Uat = at<float>(ctx, P.uat);
  float* Ugt = at<float>(ctx, P.ugt);
  float* T = at<float>(ctx, P.t);
  float* Mt = at<float>(ctx, P.mt);
  float* T2t = at<float>(ctx, P.t2);
  if (r_a > 0) {  // T = J U_a diag(c_a), through U_a^T
    STAGE(ctx, ST_APPLY_T);
    CK(transpose_f32(U_a, ld_ua, d_a, r_a, Uat, P.ld_uat, s));
    GemmDesc<float> g = {};
    g.M = d_g; g.N = r_a; g.K = d_a;
    g.A = J; g.sam = ldj; g.sak = 1;
    g.B = Uat; g.sbn = P.ld_uat; g.sbk = 1;
    g.D = T; g.ldd = P.ld_t;
    g.alpha = 1.0f; g.colscale = coef_a; g.zsplit = 1;
    g.ws = at<float>(ctx, P.ws); g.ws_floats = P.ws_floats;
    g.flags = ctx->dflags; g.wait_cycles = ctx->wait_cycles; g.split_target = ctx->split_target;
    CK(tail(g, true, J, ldj, d_g, d_a, P.big_lo, P.ld_jp));
    CK(tail(g, false, Uat, P.ld_uat, r_a, d_a, P.uat_lo, P.ld_uat));
    CK(gemm_f32(g, prec, s));
  }
  {  // M^T = U_a T^T + J^T / lambda
    STAGE(ctx, ST_APPLY_M);
    GemmDesc<float> g = {};
    g.M = d_a; g.N = d_g; g.K = r_a;
    g.A = U_a; g.sam = r_a > 0 ? ld_ua : 1; g.sak = 1;
    g.B = T; g.sbn = P.ld_t; g.sbk = 1;
    g.D = Mt; g.ldd = P.ld_mt;
    g.alpha = 1.0f; g.beta = inv_lam; g.C0 = J; g.ldc = ldj; g.c0_trans = 1; g.zsplit = 1;
    g.flags = ctx->dflags; g.wait_cycles = ctx->wait_cycles; g.split_target = ctx->split_target;
    if (r_a > 0) {
      CK(tail(g, true, U_a, ld_ua, d_a, r_a, P.ua_lo, P.ld_uap));
      CK(tail(g, false, T, P.ld_t, d_g, r_a, P.t_lo, P.ld_t));
    }
    CK(gemm_f32(g, prec, s));
  }
  if (r_g > 0) {  // T2^T = M^T U_g diag(c_g), through U_g^T
    STAGE(ctx, ST_APPLY_T2);
    CK(transpose_f32(U_g, ld_ug, d_g, r_g, Ugt, P.ld_ugt, s));
    GemmDesc<float> g = {};
    g.M = d_a; g.N = r_g; g.K = d_g;
    g.A = Mt; g.sam = P.ld_mt; g.sak = 1;
    g.B = Ugt; g.sbn = P.ld_ugt; g.sbk = 1;
    g.D = T2t; g.ldd = P.ld_t2;
    g.alpha = 1.0f; g.colscale = coef_g; g.zsplit = 1;
    g.ws = at<float>(ctx, P.ws); g.ws_floats = P.ws_floats;
    g.flags = ctx->dflags; g.wait_cycles = ctx->wait_cycles; g.split_target = ctx->split_target;
    CK(tail(g, true, Mt, P.ld_mt, d_a, d_g, P.big_lo, P.ld_mt));  // J's tails are dead: the plane is reused
    CK(tail(g, false, Ugt, P.ld_ugt, r_g, d_g, P.ugt_lo, P.ld_ugt));
    CK(gemm_f32(g, prec, s));
  }
  {  // S = U_g T2 + M / lambda  (M read through M^T)
    STAGE(ctx, ST_APPLY_S);
    GemmDesc<float> g = {};
    g.M = d_g; g.N = d_a; g.K = r_g;
    g.A = U_g; g.sam = r_g > 0 ? ld_ug : 1; g.sak = 1;
    g.B = T2t; g.sbn = P.ld_t2; g.sbk = 1;
    g.D = S; g.ldd = lds;
    g.alpha = 1.0f; g.beta = inv_lam; g.C0 = Mt; g.ldc = P.ld_mt; g.c0_trans = 1; g.zsplit = 1;
    g.flags = ctx->dflags; g.wait_cycles = ctx->wait_cycles; g.split_target = ctx->split_target;
    if (r_g > 0) {
      CK(tail(g, true, U_g, ld_ug, d_g, r_g, P.ug_lo, P.ld_ugp));
      CK(tail(g, false, T2t, P.ld_t2, d_a, r_g, P.t2_lo, P.ld_t2));
    }
    CK(gemm_f32(g, prec, s));
  }
  return KFAC_OK;
}

// Stream assignment of a grouped call: jobs are taken longest first and each
// goes to the stream with the least estimated work so far (longest processing
// time first). order: enqueue order (longest first); slot[f]: stream of job f.
void lpt_schedule(const std::vector<double>& cost, int ns, std::vector<int>& order, std::vector<int>& slot) {
  const int n = (int)cost.size();
  order.resize(n);
  slot.assign(n, 0);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<double> load(std::max(ns, 1), 0.0);
  for (int f : order) {
    const int q = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    slot[f] = q;
    load[q] += cost[f];
  }
}

// Per-stream workspace bases for a grouped call: stream q gets a slice as large
// as the largest job assigned to it.
std::vector<size_t> stream_bases(const std::vector<size_t>& need, const std::vector<int>& slot, int ns) {
  std::vector<size_t> m(ns, 0), base(ns + 1, 0);
  for (size_t f = 0; f < need.size(); ++f) m[slot[f]] = std::max(m[slot[f]], need[f]);
  for (int q = 0; q < ns; ++q) base[q + 1] = base[q] + ((m[q] + 255) & ~size_t(255));
  return base;
}

// Estimated device seconds of one randomized inversion: the large products at
// ~100 TFLOP/s plus the latency-bound k x k chain (~3 ms at k = 230, growing
// as k^2).
double invert_cost(const kfac_invert_desc& a) {
  const double d = a.d, k = (double)a.rank + a.oversample;
  if (k >= d) return 1e-3 * (d / 230.0) * (d / 230.0);
  return (a.power_iters + 2) * 2.0 * d * d * k / 1e14 + 3e-3 * (k / 230.0) * (k / 230.0);
}

// Per-item status words for a grouped call of `count` items (allocated before
// anything is enqueued, so a captured grouped call needs an earlier call with
// at least as many items).
kfac_status ensure_items(kfac_ctx* ctx, int count) {
  if (count > ctx->item_cap) {
    if (ctx->ditems) {
      if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return KFAC_ERR_CUDA;
      cudaFree(ctx->ditems);
      ctx->ditems = nullptr;
      ctx->item_cap = 0;
    }
    const int cap = std::max(count, 64);
    if (cudaMalloc(&ctx->ditems, sizeof(int) * (size_t)cap) != cudaSuccess) {
      cudaGetLastError();
      return KFAC_ERR_OOM;
    }
    if (cudaMemset(ctx->ditems, 0, sizeof(int) * (size_t)cap) != cudaSuccess) return KFAC_ERR_CUDA;
    ctx->item_cap = cap;
  }
  ctx->item_used = std::max(ctx->item_used, count);
  return KFAC_OK;
}

kfac_status ensure_side_streams(kfac_ctx* ctx, int n) {
  if (!ctx->fork_ev && cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming) != cudaSuccess)
    return KFAC_ERR_CUDA;
  for (int q = 0; q < n; ++q) {
    if (!ctx->side[q] && cudaStreamCreateWithFlags(&ctx->side[q], cudaStreamNonBlocking) != cudaSuccess)
      return KFAC_ERR_CUDA;
    if (!ctx->join_ev[q] && cudaEventCreateWithFlags(&ctx->join_ev[q], cudaEventDisableTiming) != cudaSuccess)
      return KFAC_ERR_CUDA;
  }
  return KFAC_OK;
}

}  // namespace

// ============================================================================
extern "C" {

KFAC_API int kfac_version(void) { return 100; }

KFAC_API const char* kfac_status_string(kfac_status st) {
  switch (st) {
    case KFAC_OK: return "KFAC_OK";
    case KFAC_ERR_INVALID_ARG: return "KFAC_ERR_INVALID_ARG";
    case KFAC_ERR_CUDA: return "KFAC_ERR_CUDA";
    case KFAC_ERR_OOM: return "KFAC_ERR_OOM";
    case KFAC_ERR_CHOLESKY: return "KFAC_ERR_CHOLESKY";
    case KFAC_ERR_NOCONVERGE: return "KFAC_ERR_NOCONVERGE";
    case KFAC_ERR_NONFINITE: return "KFAC_ERR_NONFINITE";
    case KFAC_ERR_TIMEOUT: return "KFAC_ERR_TIMEOUT";
    case KFAC_ERR_UNSUPPORTED: return "KFAC_ERR_UNSUPPORTED";
    case KFAC_ERR_TOO_LARGE: return "KFAC_ERR_TOO_LARGE";
  }
  return "KFAC_ERR_UNKNOWN";
}

KFAC_API kfac_status kfac_create(kfac_ctx** out, int device, void* stream) {
  if (!out) return KFAC_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) { cudaGetLastError(); return KFAC_ERR_CUDA; }
  if (device < 0 || device >= ndev) return KFAC_ERR_INVALID_ARG;
  DeviceGuard g(device);
  if (!g.ok) return KFAC_ERR_CUDA;
  kfac_ctx* ctx = new (std::nothrow) kfac_ctx();
  if (!ctx) return KFAC_ERR_OOM;
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(stream);
  if (cudaMalloc(&ctx->dflags, 64) != cudaSuccess) {
    delete ctx;
    return KFAC_ERR_OOM;
  }
  ctx->dglobal = ctx->dflags;
  ctx->dstats = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(ctx->dflags) + 32);
  if (cudaMemset(ctx->dflags, 0, 64) != cudaSuccess) {
    cudaFree(ctx->dflags);
    delete ctx;
    return KFAC_ERR_CUDA;
  }
  *out = ctx;
  return KFAC_OK;
}

KFAC_API kfac_status kfac_destroy(kfac_ctx* ctx) {
  if (!ctx) return KFAC_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (int q = 0; q < kMaxSideStreams; ++q) {
    if (ctx->side[q]) { cudaStreamSynchronize(ctx->side[q]); cudaStreamDestroy(ctx->side[q]); }
    if (ctx->join_ev[q]) cudaEventDestroy(ctx->join_ev[q]);
  }
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  for (cudaEvent_t e : ctx->item_ev) cudaEventDestroy(e);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->ditems) cudaFree(ctx->ditems);
  if (ctx->dglobal) cudaFree(ctx->dglobal);
  delete ctx;
  return KFAC_OK;
}

KFAC_API kfac_status kfac_set_stream(kfac_ctx* ctx, void* stream) {
  if (!ctx) return KFAC_ERR_INVALID_ARG;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return KFAC_OK;
}

KFAC_API kfac_status kfac_set_option(kfac_ctx* ctx, kfac_option opt, double v) {
  if (!ctx) return KFAC_ERR_INVALID_ARG;
  switch (opt) {
    case KFAC_OPT_CHOLQR_PASSES:
      if (v < 1 || v > 6) return KFAC_ERR_INVALID_ARG;
      ctx->cholqr_passes = (int)v;
      return KFAC_OK;
    case KFAC_OPT_CHOLQR_SHIFT:
      if (!(v >= 0 && v < 1)) return KFAC_ERR_INVALID_ARG;
      ctx->cholqr_shift = v;
      return KFAC_OK;
    case KFAC_OPT_EIG_REFINE:
      if (v < 0 || v > 3) return KFAC_ERR_INVALID_ARG;
      ctx->eig_refine = (int)v;
      return KFAC_OK;
    case KFAC_OPT_EIG_MAX_SWEEPS:
      if (v < 1 || v > 1000) return KFAC_ERR_INVALID_ARG;
      ctx->eig_max_sweeps = (int)v;
      return KFAC_OK;
    case KFAC_OPT_EIG_TOL:
      if (!(v > 0 && v < 1)) return KFAC_ERR_INVALID_ARG;
      ctx->eig_tol = v;
      return KFAC_OK;
    case KFAC_OPT_CHOLQR_INNER_PASSES:
      if (v < 1 || v > 6) return KFAC_ERR_INVALID_ARG;
      ctx->cholqr_inner_passes = (int)v;
      return KFAC_OK;
    case KFAC_OPT_CHOLQR_INNER_FP32:
      if (v != 0 && v != 1) return KFAC_ERR_INVALID_ARG;
      ctx->cholqr_inner_fp32 = (int)v;
      return KFAC_OK;
    case KFAC_OPT_BASIS_POLISH:
      if (v != 0 && v != 1) return KFAC_ERR_INVALID_ARG;
      ctx->basis_polish = (int)v;
      return KFAC_OK;
    case KFAC_OPT_CHOLQR_FP32_PASSES:
      if (v < 0 || v > 6) return KFAC_ERR_INVALID_ARG;
      ctx->cholqr_fp32_passes = (int)v;
      return KFAC_OK;
    case KFAC_OPT_EIG_STOP_TOL:
      if (!(v >= 0 && v < 1)) return KFAC_ERR_INVALID_ARG;
      ctx->eig_stop_tol = v;
      return KFAC_OK;
    case KFAC_OPT_EIG_REFINE_FP64:
      if (v != 0 && v != 1) return KFAC_ERR_INVALID_ARG;
      ctx->eig_refine_fp64 = (int)v;
      return KFAC_OK;
    case KFAC_OPT_CONV_CHUNK:
      if (!(v >= 1 && v <= 1e10)) return KFAC_ERR_INVALID_ARG;
      ctx->conv_chunk = (long long)v;
      return KFAC_OK;
    case KFAC_OPT_WARM_START:
      if (v != 0 && v != 1) return KFAC_ERR_INVALID_ARG;
      ctx->warm_start = (int)v;
      return KFAC_OK;
    case KFAC_OPT_SPLIT_TARGET:
      if (v < -1 || v > 4096) return KFAC_ERR_INVALID_ARG;
      ctx->split_target = (int)v;
      return KFAC_OK;
    case KFAC_OPT_CHOL_PANEL:
      if (v != 16 && v != 32) return KFAC_ERR_INVALID_ARG;
      ctx->chol_panel = (int)v;
      return KFAC_OK;
    case KFAC_OPT_TAIL_PLANES:
      if (v != 0 && v != 1) return KFAC_ERR_INVALID_ARG;
      ctx->tail_planes = (int)v;
      return KFAC_OK;
    case KFAC_OPT_CHOL_BLOCKED:
      if (v != 0 && v != 1) return KFAC_ERR_INVALID_ARG;
      ctx->chol_blocked = (int)v;
      return KFAC_OK;
    case KFAC_OPT_TRSM_INVERSE:
      if (v != 0 && v != 1) return KFAC_ERR_INVALID_ARG;
      ctx->trsm_inverse = (int)v;
      return KFAC_OK;
    case KFAC_OPT_CHOL_CLUSTER:
      if (v < 0 || v > 16) return KFAC_ERR_INVALID_ARG;
      ctx->chol_cluster = (int)v;
      return KFAC_OK;
    case KFAC_OPT_INVERT_METHOD:
      if (v != 0 && v != 1) return KFAC_ERR_INVALID_ARG;
      ctx->invert_method = (int)v;
      return KFAC_OK;
    case KFAC_OPT_GROUP_STREAMS:
      if (v < 1 || v > kMaxSideStreams) return KFAC_ERR_INVALID_ARG;
      ctx->group_streams = (int)v;
      return KFAC_OK;
    case KFAC_OPT_WAIT_CYCLES:
      if (!(v >= 1 && v <= 1e12)) return KFAC_ERR_INVALID_ARG;
      ctx->wait_cycles = (long long)v;
      return KFAC_OK;
  }
  return KFAC_ERR_INVALID_ARG;
}

KFAC_API kfac_status kfac_reserve(kfac_ctx* ctx, int d_max, int k_max, int64_t mn_max) {
  if (!ctx || d_max < 0 || k_max < 0 || mn_max < 0) return KFAC_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  size_t need = 0;
  if (d_max > 0 && k_max > 0) {
    InvertLayout a = invert_layout(d_max, std::min(k_max, d_max - 1 > 0 ? d_max - 1 : 1), k_max, true, true);
    InvertLayout a2 = invert_layout(d_max, std::min(k_max, d_max - 1 > 0 ? d_max - 1 : 1), k_max, true, false, true);
    InvertLayout b = invert_layout(std::min(d_max, k_max), k_max, k_max, true);
    a.total = std::max(a.total, a2.total);
    need = std::max(a.total, b.total);
  }
  if (mn_max > 0) {  // preconditioner apply: M^T (and a padded copy of J, a tail plane) plus thin intermediates
                     // (and their tails) and split-K partials
    const size_t dk = (size_t)std::max(d_max, 1) * (std::max(k_max, 1) + 4);
    const size_t mn_pad = (size_t)mn_max + 4 * (size_t)std::max(d_max, 1);
    size_t p = sizeof(float) * (3 * mn_pad + (12 + kApplyMaxSplit) * dk) + 20 * 256;
    need = std::max(need, p);
  }
  return ensure_ws(ctx, need);
}

KFAC_API kfac_status kfac_gemm_nt(kfac_ctx* ctx, int M, int N, int K, const float* A, int lda, const float* B,
                                  int ldb, float alpha, float beta, float* D, int ldd, kfac_precision prec) {
  if (!ctx || M < 0 || N < 0 || K < 0 || prec < KFAC_PREC_FP32 || prec > KFAC_PREC_BF16) return KFAC_ERR_INVALID_ARG;
  if ((long long)M * N == 0) return KFAC_OK;
  if (!D || ldd < N || (K > 0 && (!A || !B || lda < K || ldb < K))) return KFAC_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return KFAC_ERR_CUDA;
  const long long ws_floats = std::min<long long>(6LL * M * N, 1LL << 24);
  const long long kp = round_up(K, 4);
  const bool pack_a = K > 0 && !tma_rows_ok(A, lda), pack_b = K > 0 && !tma_rows_ok(B, ldb);
  Bump b;
  const size_t o_ws = b.take<float>((size_t)ws_floats);
  const size_t o_a = pack_a ? b.take<float>((size_t)M * kp) : 0;
  const size_t o_b = pack_b ? b.take<float>((size_t)N * kp) : 0;
  const bool tails = ctx->tail_planes != 0 && prec == KFAC_PREC_FP32 && K > 0;
  const size_t o_alo = tails ? b.take<float>((size_t)M * kp) : 0;
  const size_t o_blo = tails ? b.take<float>((size_t)N * kp) : 0;
  kfac_status st = ensure_ws(ctx, b.off);
  if (st != KFAC_OK) return st;
  if (pack_a) {  // rows TMA cannot read: the tensor-core kernel reads padded copies
    CK(pack_rows_f32(A, lda, M, K, at<float>(ctx, o_a), kp, ctx->stream));
    A = at<float>(ctx, o_a);
    lda = (int)kp;
  }
  if (pack_b) {
    CK(pack_rows_f32(B, ldb, N, K, at<float>(ctx, o_b), kp, ctx->stream));
    B = at<float>(ctx, o_b);
    ldb = (int)kp;
  }
  GemmDesc<float> g = {};
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.sam = lda; g.sak = 1;
  g.B = B; g.sbn = ldb; g.sbk = 1;
  g.D = D; g.ldd = ldd;
  g.alpha = alpha; g.beta = beta; g.C0 = D; g.ldc = ldd;
  g.zsplit = 1; g.ws = at<float>(ctx, o_ws); g.ws_floats = ws_floats;
  g.flags = ctx->dflags; g.wait_cycles = ctx->wait_cycles; g.split_target = ctx->split_target;
  if (tails && tma_rows_ok(A, lda) && tma_rows_ok(B, ldb)) {
    CK(tails_f32(A, lda, M, K, at<float>(ctx, o_alo), kp, ctx->stream));
    CK(tails_f32(B, ldb, N, K, at<float>(ctx, o_blo), kp, ctx->stream));
    g.A_lo = at<float>(ctx, o_alo); g.ld_alo = kp;
    g.B_lo = at<float>(ctx, o_blo); g.ld_blo = kp;
  }
  CK(gemm_f32(g, prec, ctx->stream));
  return KFAC_OK;
}

KFAC_API kfac_status kfac_get_status(kfac_ctx* ctx, int* flags) {
  if (!ctx) return KFAC_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  int h = 0;
  std::vector<int> items((size_t)ctx->item_used);
  if (cudaMemcpyAsync(&h, ctx->dglobal, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
    return KFAC_ERR_CUDA;
  if (ctx->item_used > 0 && cudaMemcpyAsync(items.data(), ctx->ditems, sizeof(int) * items.size(),
                                            cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
    return KFAC_ERR_CUDA;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return KFAC_ERR_CUDA;
  if (cudaMemsetAsync(ctx->dglobal, 0, sizeof(int), ctx->stream) != cudaSuccess) return KFAC_ERR_CUDA;
  if (ctx->item_used > 0 &&
      cudaMemsetAsync(ctx->ditems, 0, sizeof(int) * (size_t)ctx->item_used, ctx->stream) != cudaSuccess)
    return KFAC_ERR_CUDA;
  for (int v : items) h |= v;
  if (flags) *flags = h;
  if (h & KFAC_FLAG_NONFINITE) return KFAC_ERR_NONFINITE;
  if (h & KFAC_FLAG_CHOL_FAILED) return KFAC_ERR_CHOLESKY;
  if (h & KFAC_FLAG_EIG_NOCONV) return KFAC_ERR_NOCONVERGE;
  if (h & KFAC_FLAG_TIMEOUT) return KFAC_ERR_TIMEOUT;
  return KFAC_OK;
}

// Workspace bytes of one EA update: a padded copy of X when TMA cannot read its rows.
static bool ea_tails(const kfac_ctx* ctx, int n, kfac_precision prec) {
  return ctx->tail_planes != 0 && n > 0 && prec == KFAC_PREC_FP32;
}

static size_t ea_ws_bytes(const kfac_ctx* ctx, int d, int n, const float* X, int ldx, kfac_precision prec) {
  const size_t plane = sizeof(float) * (size_t)d * (size_t)round_up(std::max(n, 1), 4) + 256;
  return (n > 0 && !tma_rows_ok(X, ldx) ? plane : 0) + (ea_tails(ctx, n, prec) ? plane : 0);
}

// One EA update on ctx->stream; from byte offset `base` of the workspace a
// ragged X is first packed and its 3xTF32 tails formed.
static kfac_status ea_run(kfac_ctx* ctx, int d, int n, const float* X, int ldx, float rho, kfac_precision prec,
                          float* F, int ldf, size_t base) {
  STAGE(ctx, ST_EA);
  const long long ldp = round_up(std::max(n, 1), 4);
  const size_t plane = sizeof(float) * (size_t)d * (size_t)ldp + 256;
  size_t off = (base + 255) & ~size_t(255);
  if (n > 0 && !tma_rows_ok(X, ldx)) {
    float* Xp = at<float>(ctx, off);
    CK(pack_rows_f32(X, ldx, d, n, Xp, ldp, ctx->stream));
    X = Xp;
    ldx = (int)ldp;
    off = (off + plane + 255) & ~size_t(255);
  }
  float* lo = nullptr;
  if (ea_tails(ctx, n, prec)) {
    lo = at<float>(ctx, off);
    CK(tails_f32(X, ldx, d, n, lo, ldp, ctx->stream));
  }
  CK(ea_syrk(ctx->stream, d, n, X, ldx, rho, prec, F, ldf, ctx->dflags, ctx->wait_cycles, lo, ldp));
  return KFAC_OK;
}

KFAC_API kfac_status kfac_get_item_status(kfac_ctx* ctx, int count, int* item_flags) {
  if (!ctx || count < 0 || (count > 0 && !item_flags)) return KFAC_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  for (int i = 0; i < count; ++i) item_flags[i] = 0;
  const int n = std::min(count, ctx->item_used);
  if (n > 0 && cudaMemcpyAsync(item_flags, ctx->ditems, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost,
                               ctx->stream) != cudaSuccess)
    return KFAC_ERR_CUDA;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return KFAC_ERR_CUDA;
  return KFAC_OK;
}

KFAC_API kfac_status kfac_ea_update(kfac_ctx* ctx, int d, int n, const float* X, int ldx, float rho,
                                    kfac_precision prec, float* F, int ldf) {
  if (!ctx || d < 0 || n < 0 || ldf < d || (d > 0 && !F) || (n > 0 && (!X || ldx < n))) return KFAC_ERR_INVALID_ARG;
  if (!(rho >= 0.0f && rho <= 1.0f) || prec < KFAC_PREC_FP32 || prec > KFAC_PREC_BF16) return KFAC_ERR_INVALID_ARG;
  if (d == 0) return KFAC_OK;
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return KFAC_ERR_CUDA;
  kfac_status st = ensure_ws(ctx, ea_ws_bytes(ctx, d, n, X, ldx, prec));
  if (st != KFAC_OK) return st;
  return ea_run(ctx, d, n, X, ldx, rho, prec, F, ldf, 0);
}

KFAC_API kfac_status kfac_ea_update_rows(kfac_ctx* ctx, int n, int cols, const float* A, int lda, int append_one,
                                         float scale, float rho, kfac_precision prec, float* F, int ldf) {
  const int d = cols + (append_one ? 1 : 0);
  if (!ctx || n < 0 || cols < 0 || d == 0 || ldf < d || !F || (n > 0 && cols > 0 && (!A || lda < cols)))
    return KFAC_ERR_INVALID_ARG;
  if (!(rho >= 0.0f && rho <= 1.0f) || !(scale == scale) || prec < KFAC_PREC_FP32 || prec > KFAC_PREC_BF16)
    return KFAC_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return KFAC_ERR_CUDA;
  const long long ldx = round_up(std::max(n, 1), 4);
  const size_t xbytes = (sizeof(float) * (size_t)d * (size_t)ldx + 255) & ~size_t(255);
  kfac_status st = ensure_ws(ctx, xbytes + ea_ws_bytes(ctx, d, n, nullptr, (int)ldx, prec));
  if (st != KFAC_OK) return st;
  float* X = at<float>(ctx, 0);
  {
    STAGE(ctx, ST_TRANSPOSE);
    CK(rows_to_cols_f32(A, lda, n, cols, append_one ? 1 : 0, scale, X, ldx, ctx->stream));
  }
  return ea_run(ctx, d, n, X, (int)ldx, rho, prec, F, ldf, xbytes);
}

KFAC_API kfac_status kfac_ea_update_conv(kfac_ctx* ctx, int n, int c, int h, int w, const float* x, int kh, int kw,
                                         int stride_h, int stride_w, int pad_h, int pad_w, int append_one, float scale,
                                         float rho, kfac_precision prec, float* F, int ldf) {
  if (!ctx || n < 0 || c <= 0 || h <= 0 || w <= 0 || kh <= 0 || kw <= 0 || stride_h <= 0 || stride_w <= 0 ||
      pad_h < 0 || pad_w < 0 || kh > h + 2 * pad_h || kw > w + 2 * pad_w)
    return KFAC_ERR_INVALID_ARG;
  const long long dl = (long long)c * kh * kw + (append_one ? 1 : 0);
  if (!F || ldf < dl || (n > 0 && !x)) return KFAC_ERR_INVALID_ARG;
  if (dl > 65535) return KFAC_ERR_UNSUPPORTED;  // one grid row of the patch kernel per factor row
  if (!(rho >= 0.0f && rho <= 1.0f) || !(scale == scale) || prec < KFAC_PREC_FP32 || prec > KFAC_PREC_BF16)
    return KFAC_ERR_INVALID_ARG;
  const int d = (int)dl;
  const int ho = (h + 2 * pad_h - kh) / stride_h + 1, wo = (w + 2 * pad_w - kw) / stride_w + 1;
  const long long pos = (long long)ho * wo;
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return KFAC_ERR_CUDA;
  // Samples per chunk: the patch matrix of a chunk fits KFAC_OPT_CONV_CHUNK floats.
  long long per = std::max<long long>(1, ctx->conv_chunk / std::max<long long>(1, (long long)d * pos));
  per = std::min<long long>(per, std::max(n, 1));
  while (per > 1 && per * pos > (1LL << 30)) per /= 2;
  const long long ldx = round_up(per * pos, 4);
  const size_t xbytes = (sizeof(float) * (size_t)d * (size_t)ldx + 255) & ~size_t(255);
  const bool tails = ea_tails(ctx, n, prec);
  kfac_status st = ensure_ws(ctx, xbytes * (tails ? 2 : 1));
  if (st != KFAC_OK) return st;
  float* X = at<float>(ctx, 0);
  float* Xlo = tails ? at<float>(ctx, xbytes) : nullptr;
  const float alpha = n > 0 ? (1.0f - rho) / (float)((double)n * pos) : 0.0f;
  STAGE(ctx, ST_EA);
  if (n == 0) {
    CK(syrk_update(ctx->stream, d, 0, X, (int)ldx, 0.0f, rho, prec, F, ldf, ctx->dflags, ctx->wait_cycles));
    return KFAC_OK;
  }
  for (int i0 = 0; i0 < n; i0 += (int)per) {
    const int ns = (int)std::min<long long>(per, n - i0);
    CK(im2col_f32(x, c, h, w, kh, kw, stride_h, stride_w, pad_h, pad_w, i0, ns, append_one ? 1 : 0, scale, X, ldx,
                  ctx->stream));
    if (Xlo) CK(tails_f32(X, ldx, d, (int)(ns * pos), Xlo, ldx, ctx->stream));
    CK(syrk_update(ctx->stream, d, (int)(ns * pos), X, (int)ldx, alpha, i0 == 0 ? rho : 1.0f, prec, F, ldf,
                   ctx->dflags, ctx->wait_cycles, Xlo, ldx));
  }
  return KFAC_OK;
}

static kfac_status check_ea(const kfac_ea_desc& a) {
  if (a.d < 0 || a.n < 0 || a.ldf < a.d || (a.d > 0 && !a.F) || (a.n > 0 && (!a.X || a.ldx < a.n)))
    return KFAC_ERR_INVALID_ARG;
  if (!(a.rho >= 0.0f && a.rho <= 1.0f) || a.prec < KFAC_PREC_FP32 || a.prec > KFAC_PREC_BF16)
    return KFAC_ERR_INVALID_ARG;
  return KFAC_OK;
}

KFAC_API kfac_status kfac_ea_update_grouped(kfac_ctx* ctx, int count, const kfac_ea_desc* descs) {
  if (!ctx || count < 0 || (count > 0 && !descs)) return KFAC_ERR_INVALID_ARG;
  for (int f = 0; f < count; ++f) {
    kfac_status st = check_ea(descs[f]);
    if (st != KFAC_OK) return st;
  }
  if (count == 0) return KFAC_OK;
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return KFAC_ERR_CUDA;
  const int ns = std::min(count, ctx->group_streams);
  std::vector<double> cost(count);
  std::vector<size_t> need(count);  // padded copies of ragged X
  for (int f = 0; f < count; ++f) {
    const kfac_ea_desc& a = descs[f];
    cost[f] = (double)a.d * a.d * (a.n + 8);
    need[f] = ea_ws_bytes(ctx, a.d, a.n, a.X, a.ldx, a.prec);
  }
  std::vector<int> order, slot;
  lpt_schedule(cost, ns, order, slot);
  const std::vector<size_t> base = stream_bases(need, slot, ns);
  kfac_status st = ensure_ws(ctx, base[ns]);
  if (st != KFAC_OK) return st;
  if ((st = ensure_items(ctx, count)) != KFAC_OK) return st;
  if (ns > 1 && (st = ensure_side_streams(ctx, ns)) != KFAC_OK) return st;
  cudaStream_t main_s = ctx->stream;
  if (ns > 1) {
    CK(cudaEventRecord(ctx->fork_ev, main_s));
    for (int q = 0; q < ns; ++q) CK(cudaStreamWaitEvent(ctx->side[q], ctx->fork_ev, 0));
  }
  kfac_status first_err = KFAC_OK;
  for (int i = 0; i < count && first_err == KFAC_OK; ++i) {
    const int f = order[i];
    const kfac_ea_desc& a = descs[f];
    if (a.d == 0) continue;
    ctx->stream = ns > 1 ? ctx->side[slot[f]] : main_s;
    ctx->dflags = ctx->ditems + f;
    first_err = ea_run(ctx, a.d, a.n, a.X, a.ldx, a.rho, a.prec, a.F, a.ldf, base[slot[f]]);
  }
  ctx->dflags = ctx->dglobal;
  ctx->stream = main_s;
  if (ns > 1) {
    for (int q = 0; q < ns; ++q) {
      CK(cudaEventRecord(ctx->join_ev[q], ctx->side[q]));
      CK(cudaStreamWaitEvent(main_s, ctx->join_ev[q], 0));
    }
  }
  return first_err;
}

KFAC_API kfac_status kfac_rsvd_invert(kfac_ctx* ctx, int d, const float* F, int ldf, int rank, int oversample,
                                      int power_iters, float lambda, const float* omega, int ldo,
                                      unsigned long long seed, kfac_precision prec, float* U, int ldu, float* D,
                                      float* coef) {
  if (!ctx) return KFAC_ERR_INVALID_ARG;
  kfac_invert_desc a = {d, F, ldf, rank, oversample, power_iters, lambda, omega, ldo, prec, U, ldu, D, coef, seed};
  int r = 0, k = 0;
  kfac_status st = check_invert(a, &r, &k);
  if (st != KFAC_OK) return st;
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return KFAC_ERR_CUDA;
  InvertLayout L = invert_layout(d, k, r, !tma_rows_ok(F, ldf), prec == KFAC_PREC_BF16, ctx->tail_planes != 0);
  if ((st = ensure_ws(ctx, L.total)) != KFAC_OK) return st;
  return invert_run(ctx, a, L, 0);
}

KFAC_API kfac_status kfac_draw_omega(kfac_ctx* ctx, int d, int k, unsigned long long seed, float* omega, int ldo) {
  if (!ctx || d < 1 || k < 1 || !omega || ldo < k) return KFAC_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return KFAC_ERR_CUDA;
  return draw_omega_f32(d, k, seed, 0, k, omega, ldo, false, ctx->stream) == cudaSuccess ? KFAC_OK : KFAC_ERR_CUDA;
}

KFAC_API kfac_status kfac_rsvd_invert_grouped(kfac_ctx* ctx, int count, const kfac_invert_desc* descs) {
  if (!ctx || count < 0 || (count > 0 && !descs)) return KFAC_ERR_INVALID_ARG;
  if (count == 0) return KFAC_OK;
  std::vector<InvertLayout> lay(count);
  for (int f = 0; f < count; ++f) {
    int r = 0, k = 0;
    kfac_status st = check_invert(descs[f], &r, &k);
    if (st != KFAC_OK) return st;
    lay[f] = invert_layout(descs[f].d, k, r, !tma_rows_ok(descs[f].F, descs[f].ldf), descs[f].prec == KFAC_PREC_BF16,
                           ctx->tail_planes != 0);
  }
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return KFAC_ERR_CUDA;
  const int ns = std::min(count, ctx->group_streams);
  std::vector<double> cost(count);
  std::vector<size_t> need(count);
  for (int f = 0; f < count; ++f) {
    cost[f] = invert_cost(descs[f]);
    need[f] = lay[f].total;
  }
  std::vector<int> order, slot;
  lpt_schedule(cost, ns, order, slot);
  const std::vector<size_t> base = stream_bases(need, slot, ns);
  kfac_status st = ensure_ws(ctx, base[ns]);
  if (st != KFAC_OK) return st;
  if ((st = ensure_items(ctx, count)) != KFAC_OK) return st;
  if (count == 1) {
    ctx->dflags = ctx->ditems;
    st = invert_run(ctx, descs[0], lay[0], 0);
    ctx->dflags = ctx->dglobal;
    return st;
  }
  if ((st = ensure_side_streams(ctx, ns)) != KFAC_OK) return st;
  cudaStream_t main_s = ctx->stream;
  CK(cudaEventRecord(ctx->fork_ev, main_s));
  for (int q = 0; q < ns; ++q) CK(cudaStreamWaitEvent(ctx->side[q], ctx->fork_ev, 0));
  kfac_status first_err = KFAC_OK;
  for (int i = 0; i < count && first_err == KFAC_OK; ++i) {
    const int f = order[i];
    ctx->stream = ctx->side[slot[f]];
    ctx->dflags = ctx->ditems + f;
    first_err = invert_run(ctx, descs[f], lay[f], base[slot[f]]);
  }
  ctx->dflags = ctx->dglobal;
  ctx->stream = main_s;
  for (int q = 0; q < ns; ++q) {
    CK(cudaEventRecord(ctx->join_ev[q], ctx->side[q]));
    CK(cudaStreamWaitEvent(main_s, ctx->join_ev[q], 0));
  }
  return first_err;
}

// ---- autotuner ----------------------------------------------------------------

// Shape signature of a grouped inversion (order-independent): factor count and
// a hash of every factor's (d, k, power iterations, precision), plus the
// inversion method.
static unsigned long long invert_signature(const kfac_ctx* ctx, int count, const kfac_invert_desc* descs) {
  std::vector<unsigned long long> keys(count);
  for (int f = 0; f < count; ++f) {
    const kfac_invert_desc& a = descs[f];
    keys[f] = ((unsigned long long)a.d << 32) ^ ((unsigned long long)(a.rank + a.oversample) << 12) ^
              ((unsigned long long)a.power_iters << 4) ^ (unsigned long long)a.prec;
  }
  std::sort(keys.begin(), keys.end());
  unsigned long long h = 1469598103934665603ull ^ (unsigned long long)count ^ ((unsigned long long)ctx->invert_method << 40);
  for (unsigned long long k : keys) {  // FNV-1a over the sorted keys
    for (int b = 0; b < 8; ++b) {
      h ^= (k >> (8 * b)) & 0xffull;
      h *= 1099511628211ull;
    }
  }
  return h;
}

// Looks for "<device> <signature> <streams> <chol_cluster> <split_target> <ms>"
// in the cache file; fills cfg[3] and returns true when found.
static bool cache_lookup(const char* path, const char* dev, unsigned long long sig, int* cfg) {
  FILE* fp = fopen(path, "r");
  if (!fp) return false;
  char line[512];
  bool found = false;
  while (fgets(line, sizeof line, fp)) {
    char name[256];
    unsigned long long s = 0;
    int a = 0, b = 0, c = 0, e = 0, f = 0, h = 0;
    double ms = 0.0;
    if (sscanf(line, "%255[^|]|%llx %d %d %d %d %d %d %lf", name, &s, &a, &b, &c, &e, &f, &h, &ms) == 9 &&
        s == sig && strcmp(name, dev) == 0) {
      cfg[0] = a; cfg[1] = b; cfg[2] = c; cfg[3] = e; cfg[4] = f; cfg[5] = h;
      found = true;  // the last entry for this key wins
    }
  }
  fclose(fp);
  return found;
}

KFAC_API kfac_status kfac_autotune_invert(kfac_ctx* ctx, int count, const kfac_invert_desc* descs,
                                          const char* cache_path, int* chosen) {
  if (!ctx || count <= 0 || !descs) return KFAC_ERR_INVALID_ARG;
  for (int f = 0; f < count; ++f) {
    int r = 0, k = 0;
    kfac_status st = check_invert(descs[f], &r, &k);
    if (st != KFAC_OK) return st;
  }
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return KFAC_ERR_CUDA;
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, ctx->device));
  for (char* c = prop.name; *c; ++c)
    if (*c == '|' || *c == '\n') *c = ' ';
  const unsigned long long sig = invert_signature(ctx, count, descs);
  int cfg[6] = {ctx->group_streams, ctx->chol_cluster, ctx->split_target, ctx->chol_panel, ctx->chol_blocked,
                ctx->trsm_inverse};
  bool cached = cache_path && cache_lookup(cache_path, prop.name, sig, cfg);
  cfg[5] = ctx->trsm_inverse;  // the solve form stays as set, whatever a cached line holds
  double best_ms = 0.0;
  if (!cached) {
    bool big_k = false;
    for (int f = 0; f < count; ++f) {
      const int k = descs[f].rank + descs[f].oversample;
      if (k > 236 && k < descs[f].d) big_k = true;
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return KFAC_ERR_CUDA; }
    // One warm-up and two timed grouped inversions per candidate.
    auto run = [&](const int* c, double* ms) -> kfac_status {
      ctx->group_streams = c[0]; ctx->chol_cluster = c[1]; ctx->split_target = c[2]; ctx->chol_panel = c[3];
      ctx->chol_blocked = c[4]; ctx->trsm_inverse = c[5];
      kfac_status st = kfac_rsvd_invert_grouped(ctx, count, descs);
      if (st != KFAC_OK) return st;
      if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) return KFAC_ERR_CUDA;
      for (int it = 0; it < 2 && st == KFAC_OK; ++it) st = kfac_rsvd_invert_grouped(ctx, count, descs);
      if (st != KFAC_OK) return st;
      if (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
        return KFAC_ERR_CUDA;
      float t = 0.0f;
      if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) return KFAC_ERR_CUDA;
      *ms = t / 2.0;
      return KFAC_OK;
    };
    // Coordinate descent over the knobs, from the current settings: streams,
    // blocked or cluster Cholesky, split target, then the cluster kernel's
    // size and panel width if it is in use. The solve form is left as set: the
    // explicit inverse is faster on some GPUs but less robust (its inverse of
    // a nearly singular factor can overflow), a choice for the caller.
    const int streams_c[] = {4, 8, 16, 32};
    const int chol_c[] = {0, 8, 12};
    const int split_c[] = {0, 304, -1};
    const int panel_c[] = {16, 32};
    const int blocked_c[] = {1, 0};
    const int inverse_c[] = {1, 0};
    const int order[5] = {0, 4, 2, 1, 3};
    kfac_status st = run(cfg, &best_ms);
    for (int oi = 0; oi < 5 && st == KFAC_OK; ++oi) {
      const int dim = order[oi];
      const int* cand = dim == 0 ? streams_c
                                 : (dim == 1 ? chol_c
                                             : (dim == 2 ? split_c : (dim == 3 ? panel_c : (dim == 4 ? blocked_c
                                                                                                     : inverse_c))));
      const int n = dim == 0 ? 4 : ((dim == 3 || dim == 4 || dim == 5) ? 2 : 3);
      if ((dim == 1 || dim == 3 || dim == 4) && !big_k) continue;  // no factor uses a large-order Cholesky
      if ((dim == 1 || dim == 3) && cfg[4]) continue;            // the cluster kernel is not in use
      for (int i = 0; i < n && st == KFAC_OK; ++i) {
        if (cand[i] == cfg[dim]) continue;
        int trial[6] = {cfg[0], cfg[1], cfg[2], cfg[3], cfg[4], cfg[5]};
        trial[dim] = cand[i];
        double ms = 0.0;
        st = run(trial, &ms);
        if (st == KFAC_OK && ms < best_ms) {
          best_ms = ms;
          cfg[dim] = cand[i];
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != KFAC_OK) return st;
    if (cache_path) {
      FILE* fp = fopen(cache_path, "a");
      if (fp) {
        fprintf(fp, "%s|%llx %d %d %d %d %d %d %.4f\n", prop.name, sig, cfg[0], cfg[1], cfg[2], cfg[3], cfg[4], cfg[5],
                best_ms);
        fclose(fp);
      }
    }
  }
  ctx->group_streams = cfg[0];
  ctx->chol_cluster = cfg[1];
  ctx->split_target = cfg[2];
  ctx->chol_panel = cfg[3];
  ctx->chol_blocked = cfg[4];
  ctx->trsm_inverse = cfg[5];
  if (chosen) {
    for (int i = 0; i < 6; ++i) chosen[i] = cfg[i];
    chosen[6] = cached ? 1 : 0;
  }
  return KFAC_OK;
}

KFAC_API kfac_status kfac_precondition(kfac_ctx* ctx, int d_g, int d_a, const float* J, int ldj,
                                       const float* U_a, int ld_ua, const float* coef_a, int r_a,
                                       const float* U_g, int ld_ug, const float* coef_g, int r_g,
                                       float lambda, kfac_precision prec, float* S, int lds) {
  if (!ctx || d_g < 0 || d_a < 0 || r_a < 0 || r_g < 0 || r_a > d_a || r_g > d_g) return KFAC_ERR_INVALID_ARG;
  if (!(lambda > 0.0f) || prec < KFAC_PREC_FP32 || prec > KFAC_PREC_BF16) return KFAC_ERR_INVALID_ARG;
  if ((long long)d_g * d_a == 0) return KFAC_OK;
  if (!J || ldj < d_a || !S || lds < d_a || S == J) return KFAC_ERR_INVALID_ARG;
  if (r_a > 0 && (!U_a || ld_ua < r_a || !coef_a)) return KFAC_ERR_INVALID_ARG;
  if (r_g > 0 && (!U_g || ld_ug < r_g || !coef_g)) return KFAC_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return KFAC_ERR_CUDA;
  PrecLayout P = prec_layout_for(d_g, d_a, J, ldj, U_a, ld_ua, r_a, U_g, ld_ug, r_g, ctx->tail_planes != 0);
  kfac_status st = ensure_ws(ctx, P.total);
  if (st != KFAC_OK) return st;
  return precondition_run(ctx, d_g, d_a, J, ldj, U_a, ld_ua, coef_a, r_a, U_g, ld_ug, coef_g, r_g, lambda, prec, S,
                          lds, P, 0);
}

static kfac_status check_precond(const kfac_precond_desc& a) {
  if (a.d_g < 0 || a.d_a < 0 || a.r_a < 0 || a.r_g < 0 || a.r_a > a.d_a || a.r_g > a.d_g) return KFAC_ERR_INVALID_ARG;
  if (!(a.lambda > 0.0f) || a.prec < KFAC_PREC_FP32 || a.prec > KFAC_PREC_BF16) return KFAC_ERR_INVALID_ARG;
  if ((long long)a.d_g * a.d_a == 0) return KFAC_OK;
  if (!a.J || a.ldj < a.d_a || !a.S || a.lds < a.d_a || a.S == a.J) return KFAC_ERR_INVALID_ARG;
  if (a.r_a > 0 && (!a.U_a || a.ld_ua < a.r_a || !a.coef_a)) return KFAC_ERR_INVALID_ARG;
  if (a.r_g > 0 && (!a.U_g || a.ld_ug < a.r_g || !a.coef_g)) return KFAC_ERR_INVALID_ARG;
  return KFAC_OK;
}

KFAC_API kfac_status kfac_precondition_grouped(kfac_ctx* ctx, int count, const kfac_precond_desc* descs) {
  if (!ctx || count < 0 || (count > 0 && !descs)) return KFAC_ERR_INVALID_ARG;
  for (int f = 0; f < count; ++f) {
    kfac_status st = check_precond(descs[f]);
    if (st != KFAC_OK) return st;
  }
  if (count == 0) return KFAC_OK;
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return KFAC_ERR_CUDA;
  std::vector<PrecLayout> lay(count);
  for (int f = 0; f < count; ++f) {
    const kfac_precond_desc& a = descs[f];
    lay[f] = prec_layout_for(a.d_g, a.d_a, a.J, a.ldj, a.U_a, a.ld_ua, a.r_a, a.U_g, a.ld_ug, a.r_g,
                             ctx->tail_planes != 0);
  }
  const int ns = std::min(count, ctx->group_streams);
  std::vector<double> cost(count);
  std::vector<size_t> need(count);
  for (int f = 0; f < count; ++f) {
    const kfac_precond_desc& a = descs[f];
    cost[f] = (double)a.d_g * a.d_a * (a.r_a + a.r_g + 8);
    need[f] = lay[f].total;
  }
  std::vector<int> order, slot;
  lpt_schedule(cost, ns, order, slot);
  const std::vector<size_t> base = stream_bases(need, slot, ns);
  kfac_status st = ensure_ws(ctx, base[ns]);
  if (st != KFAC_OK) return st;
  auto run = [&](int f, size_t off) -> kfac_status {
    const kfac_precond_desc& a = descs[f];
    if ((long long)a.d_g * a.d_a == 0) return KFAC_OK;
    return precondition_run(ctx, a.d_g, a.d_a, a.J, a.ldj, a.U_a, a.ld_ua, a.coef_a, a.r_a, a.U_g, a.ld_ug,
                            a.coef_g, a.r_g, a.lambda, a.prec, a.S, a.lds, lay[f], off);
  };
  if ((st = ensure_items(ctx, count)) != KFAC_OK) return st;
  if (count == 1) {
    ctx->dflags = ctx->ditems;
    st = run(0, 0);
    ctx->dflags = ctx->dglobal;
    return st;
  }
  if ((st = ensure_side_streams(ctx, ns)) != KFAC_OK) return st;
  cudaStream_t main_s = ctx->stream;
  CK(cudaEventRecord(ctx->fork_ev, main_s));
  for (int q = 0; q < ns; ++q) CK(cudaStreamWaitEvent(ctx->side[q], ctx->fork_ev, 0));
  kfac_status first_err = KFAC_OK;
  for (int i = 0; i < count && first_err == KFAC_OK; ++i) {
    const int f = order[i];
    ctx->stream = ctx->side[slot[f]];
    ctx->dflags = ctx->ditems + f;
    first_err = run(f, base[slot[f]]);
  }
  ctx->dflags = ctx->dglobal;
  ctx->stream = main_s;
  for (int q = 0; q < ns; ++q) {
    CK(cudaEventRecord(ctx->join_ev[q], ctx->side[q]));
    CK(cudaStreamWaitEvent(main_s, ctx->join_ev[q], 0));
  }
  return first_err;
}

// One K-FAC step of a set of layers (Alg. 1 EA updates, Alg. 3 / Alg. 2
// inversions, Alg. 4 applies) with per-item dependencies instead of a join
// between the phases: factor f's EA update and inversion run in turn on its
// forked stream, and layer l's apply starts as soon as its two factors are
// inverted, on the stream of the later of them (an event from the other), so
// applies overlap the inversions still running.
KFAC_API kfac_status kfac_step_grouped(kfac_ctx* ctx, int n_factors, const kfac_ea_desc* ea,
                                       const kfac_invert_desc* inv, int n_layers, const kfac_precond_desc* pre,
                                       const int* layer_factors) {
  if (!ctx || n_factors < 0 || n_layers < 0 || (n_factors > 0 && !inv) || (n_layers > 0 && (!pre || !layer_factors)))
    return KFAC_ERR_INVALID_ARG;
  std::vector<InvertLayout> il(n_factors);
  for (int f = 0; f < n_factors; ++f) {
    int r = 0, k = 0;
    kfac_status st = check_invert(inv[f], &r, &k);
    if (st != KFAC_OK) return st;
    if (ea && (st = check_ea(ea[f])) != KFAC_OK) return st;
    il[f] = invert_layout(inv[f].d, k, r, !tma_rows_ok(inv[f].F, inv[f].ldf), inv[f].prec == KFAC_PREC_BF16,
                          ctx->tail_planes != 0);
  }
  std::vector<PrecLayout> pl(n_layers);
  for (int l = 0; l < n_layers; ++l) {
    kfac_status st = check_precond(pre[l]);
    if (st != KFAC_OK) return st;
    for (int q = 0; q < 2; ++q)
      if (layer_factors[2 * l + q] < -1 || layer_factors[2 * l + q] >= n_factors) return KFAC_ERR_INVALID_ARG;
    const kfac_precond_desc& a = pre[l];
    pl[l] = prec_layout_for(a.d_g, a.d_a, a.J, a.ldj, a.U_a, a.ld_ua, a.r_a, a.U_g, a.ld_ug, a.r_g,
                            ctx->tail_planes != 0);
  }
  if (n_factors + n_layers == 0) return KFAC_OK;
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return KFAC_ERR_CUDA;
  const int ns = std::max(1, std::min(std::max(n_factors, n_layers), ctx->group_streams));
  std::vector<double> cost(n_factors);
  for (int f = 0; f < n_factors; ++f)
    cost[f] = invert_cost(inv[f]) + (ea ? 2.0 * ea[f].d * (double)ea[f].d * ea[f].n / 1e14 : 0.0);
  std::vector<int> order, slot;
  lpt_schedule(cost, ns, order, slot);
  std::vector<int> pos(n_factors, 0);
  for (int i = 0; i < n_factors; ++i) pos[order[i]] = i;
  // Each layer runs after the later (in issue order) of its factors, on that
  // factor's stream; a layer without factors runs first, spread over the streams.
  std::vector<std::vector<int>> after(n_factors);
  std::vector<int> free_layers;
  std::vector<size_t> need(n_factors + n_layers);
  std::vector<int> slot_all(n_factors + n_layers);
  for (int f = 0; f < n_factors; ++f) {
    need[f] = std::max(il[f].total, ea ? ea_ws_bytes(ctx, ea[f].d, ea[f].n, ea[f].X, ea[f].ldx, ea[f].prec) : 0);
    slot_all[f] = slot[f];
  }
  for (int l = 0; l < n_layers; ++l) {
    const int a = layer_factors[2 * l], g = layer_factors[2 * l + 1];
    const int host = a < 0 ? g : (g < 0 ? a : (pos[a] > pos[g] ? a : g));
    need[n_factors + l] = pl[l].total;
    if (host < 0) {
      free_layers.push_back(l);
      slot_all[n_factors + l] = l % ns;
    } else {
      after[host].push_back(l);
      slot_all[n_factors + l] = slot[host];
    }
  }
  const std::vector<size_t> base = stream_bases(need, slot_all, ns);
  kfac_status st = ensure_ws(ctx, base[ns]);
  if (st != KFAC_OK) return st;
  if ((st = ensure_items(ctx, n_factors + n_layers)) != KFAC_OK) return st;
  if ((st = ensure_side_streams(ctx, ns)) != KFAC_OK) return st;
  while ((int)ctx->item_ev.size() < n_factors) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return KFAC_ERR_CUDA;
    ctx->item_ev.push_back(e);
  }
  auto apply = [&](int l, int q) -> kfac_status {
    const kfac_precond_desc& a = pre[l];
    if ((long long)a.d_g * a.d_a == 0) return KFAC_OK;
    ctx->dflags = ctx->ditems + n_factors + l;
    return precondition_run(ctx, a.d_g, a.d_a, a.J, a.ldj, a.U_a, a.ld_ua, a.coef_a, a.r_a, a.U_g, a.ld_ug,
                            a.coef_g, a.r_g, a.lambda, a.prec, a.S, a.lds, pl[l], base[q]);
  };
  cudaStream_t main_s = ctx->stream;
  CK(cudaEventRecord(ctx->fork_ev, main_s));
  for (int q = 0; q < ns; ++q) CK(cudaStreamWaitEvent(ctx->side[q], ctx->fork_ev, 0));
  kfac_status first_err = KFAC_OK;
  for (int l : free_layers) {
    if (first_err != KFAC_OK) break;
    ctx->stream = ctx->side[l % ns];
    first_err = apply(l, l % ns);
  }
  for (int i = 0; i < n_factors && first_err == KFAC_OK; ++i) {
    const int f = order[i], q = slot[f];
    ctx->stream = ctx->side[q];
    ctx->dflags = ctx->ditems + f;
    if (ea && ea[f].d > 0) first_err = ea_run(ctx, ea[f].d, ea[f].n, ea[f].X, ea[f].ldx, ea[f].rho, ea[f].prec,
                                              ea[f].F, ea[f].ldf, base[q]);
    if (first_err == KFAC_OK) first_err = invert_run(ctx, inv[f], il[f], base[q]);
    if (first_err != KFAC_OK) break;
    if (cudaEventRecord(ctx->item_ev[f], ctx->stream) != cudaSuccess) { first_err = KFAC_ERR_CUDA; break; }
    for (int l : after[f]) {
      const int a = layer_factors[2 * l], g = layer_factors[2 * l + 1];
      for (int o : {a, g})
        if (o >= 0 && o != f && cudaStreamWaitEvent(ctx->stream, ctx->item_ev[o], 0) != cudaSuccess)
          first_err = KFAC_ERR_CUDA;
      if (first_err == KFAC_OK) first_err = apply(l, q);
      if (first_err != KFAC_OK) break;
    }
  }
  ctx->dflags = ctx->dglobal;
  ctx->stream = main_s;
  for (int q = 0; q < ns; ++q) {
    CK(cudaEventRecord(ctx->join_ev[q], ctx->side[q]));
    CK(cudaStreamWaitEvent(main_s, ctx->join_ev[q], 0));
  }
  return first_err;
}

KFAC_API uint64_t kfac_kernel_launch_count(void) { return (uint64_t)launch_count(); }

KFAC_API uint64_t kfac_simt_gemm_count(void) { return (uint64_t)simt_gemm_count(); }

KFAC_API kfac_status kfac_stats_read(kfac_ctx* ctx, int64_t* out, int n) {
  if (!ctx || n < 0 || (n > 0 && !out)) return KFAC_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  unsigned long long h[STAT_COUNT] = {};
  if (cudaMemcpyAsync(h, ctx->dstats, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
    return KFAC_ERR_CUDA;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return KFAC_ERR_CUDA;
  if (cudaMemsetAsync(ctx->dstats, 0, sizeof(h), ctx->stream) != cudaSuccess) return KFAC_ERR_CUDA;
  for (int i = 0; i < n && i < STAT_COUNT; ++i) out[i] = (int64_t)h[i];
  return KFAC_OK;
}

KFAC_API kfac_status kfac_profile_enable(kfac_ctx* ctx, int on) {
  if (!ctx) return KFAC_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  ctx->prof.on = on != 0;
  for (auto& u : ctx->prof.used) u = 0;
  if (ctx->prof.on) {
    if (!ctx->prof.base && cudaEventCreate(&ctx->prof.base) != cudaSuccess) return KFAC_ERR_CUDA;
    if (cudaEventRecord(ctx->prof.base, ctx->stream) != cudaSuccess) return KFAC_ERR_CUDA;
  }
  return KFAC_OK;
}

KFAC_API const char* kfac_stage_name(int stage) {
  return stage >= 0 && stage < ST_COUNT ? kStageNames[stage] : nullptr;
}

KFAC_API kfac_status kfac_profile_timeline(kfac_ctx* ctx, int max_events, int* stage, int* item, double* start_ms,
                                           double* end_ms, int* n_events) {
  if (!ctx || max_events < 0 || !ctx->prof.base) return KFAC_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return KFAC_ERR_CUDA;
  struct Iv { double a, b; int st, it; };
  std::vector<Iv> all;
  for (int i = 0; i < ST_COUNT; ++i)
    for (size_t j = 0; j < ctx->prof.used[i]; ++j) {
      float a = 0.0f, b = 0.0f;
      if (cudaEventElapsedTime(&a, ctx->prof.base, ctx->prof.ev[i][j].first) != cudaSuccess ||
          cudaEventElapsedTime(&b, ctx->prof.base, ctx->prof.ev[i][j].second) != cudaSuccess)
        return KFAC_ERR_CUDA;
      all.push_back({a, b, i, ctx->prof.item[i][j]});
    }
  std::stable_sort(all.begin(), all.end(), [](const Iv& x, const Iv& y) { return x.a < y.a; });
  const int n = std::min(max_events, (int)all.size());
  for (int e = 0; e < n; ++e) {
    if (stage) stage[e] = all[e].st;
    if (item) item[e] = all[e].it;
    if (start_ms) start_ms[e] = all[e].a;
    if (end_ms) end_ms[e] = all[e].b;
  }
  if (n_events) *n_events = (int)all.size();
  return KFAC_OK;
}

KFAC_API kfac_status kfac_profile_read(kfac_ctx* ctx, const char** names, double* total_ms, int* launches,
                                       int max_stages, int* n_stages) {
  if (!ctx || max_stages < 0) return KFAC_ERR_INVALID_ARG;
  DeviceGuard dg(ctx->device);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return KFAC_ERR_CUDA;
  int n = std::min(max_stages, (int)ST_COUNT);
  for (int i = 0; i < ST_COUNT; ++i) {
    double tot = 0.0;
    for (size_t j = 0; j < ctx->prof.used[i]; ++j) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, ctx->prof.ev[i][j].first, ctx->prof.ev[i][j].second) == cudaSuccess) tot += ms;
    }
    if (i < n) {
      if (names) names[i] = kStageNames[i];
      if (total_ms) total_ms[i] = tot;
      if (launches) launches[i] = (int)ctx->prof.used[i];
    }
    ctx->prof.used[i] = 0;
  }
  if (n_stages) *n_stages = n;
  return KFAC_OK;
}

}  // extern "C"
