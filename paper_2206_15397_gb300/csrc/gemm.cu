// GEMM-shaped steps: dispatch between the tcgen05 tensor-core kernel and the
// SIMT kernel, split-K with a reducing epilogue, and the EA SYRK.
#include "gemm.cuh"
#include "tc_gemm.cuh"

namespace kfac {
namespace {

Round round_of(kfac_precision p) {
  return p == KFAC_PREC_BF16 ? Round::BF16 : (p == KFAC_PREC_TF32 ? Round::TF32 : Round::None);
}

long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

// Sum z split-K partials (dense, in D's layout: rows x cols) and apply the
// epilogue of g, writing D.
__global__ void k_reduce_epilogue(const float* __restrict__ part, int z, long long zstride, int rows, int cols,
                                  GemmDesc<float> g) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)rows * cols) return;
  const int r = (int)(idx / cols), c = (int)(idx % cols);
  const int m = g.d_trans ? c : r, n = g.d_trans ? r : c;
  float v = 0.0f;
  for (int q = 0; q < z; ++q) v += part[q * zstride + idx];
  v *= g.alpha;
  if (g.rowscale) v *= g.rowscale[m];
  if (g.colscale) v *= g.colscale[n];
  if (g.beta != 0.0f && g.C0)
    v = fmaf(g.beta, g.C0[g.c0_trans ? (long long)n * g.ldc + m : (long long)m * g.ldc + n], v);
  g.D[(long long)r * g.ldd + c] = v;
}

}  // namespace

cudaError_t gemm_f32(const GemmDesc<float>& g, kfac_precision prec, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  const bool kmajor = g.sak == 1 && g.sbk == 1;
  const tc::Mode mode = prec == KFAC_PREC_FP32 ? tc::Mode::Fp32 : (prec == KFAC_PREC_TF32 ? tc::Mode::Tf32 : tc::Mode::Bf16);
  const int kalign = tc::k_step(mode);  // a K-chunk must cover whole K-steps of the kernel
  const bool bf16d = g.ab_bf16 != 0;     // operands already BF16: only the direct tensor-core kernel reads them
  if (bf16d && (!kmajor || g.K <= 0 || prec != KFAC_PREC_BF16 || g.sym || !tma_rows_ok(g.A, 2 * g.sam) ||
                !tma_rows_ok(g.B, 2 * g.sbn) || (g.sam & 7) || (g.sbn & 7) || g.sam < g.K || g.sbn < g.K ||
                (g.zsplit > 1 && g.kchunk % 64 != 0)))
    return cudaErrorInvalidValue;
  const bool tc_ok = bf16d || (kmajor && g.K > 0 &&
                     tc::eligible(g.A, g.sam, g.B, g.sbn, g.M, g.N, g.K) &&
                     (g.zsplit <= 1 || g.kchunk % kalign == 0));
  if (!tc_ok) {
    if (g.K > 0) note_simt_gemm();
    return gemm_simt_f32(g, round_of(prec), s);
  }
  auto launch = [&](const tc::TcArgs& a, int zsplit) {
    if (bf16d) return tc::gemm_bf16(a, g.A, g.sam, g.B, g.sbn, zsplit, s);
    const bool tails = mode == tc::Mode::Fp32;
    return tc::gemm(a, g.A, g.sam, g.B, g.sbn, zsplit, mode, s, tails ? g.A_lo : nullptr, g.ld_alo ? g.ld_alo : g.sam,
                    tails ? g.B_lo : nullptr, g.ld_blo ? g.ld_blo : g.sbn);
  };

  tc::TcArgs a = {};
  a.M = g.M; a.N = g.N; a.K = g.K;
  a.tn = tc::tile_n(g.N, mode, g.sym != 0, bf16d);
  a.alpha = g.alpha; a.beta = g.beta;
  a.rowscale = g.rowscale; a.colscale = g.colscale;
  a.C0 = g.C0; a.ldc = g.ldc; a.c0_trans = g.c0_trans;
  a.D = g.D; a.ldd = g.ldd; a.d_trans = g.d_trans;
  a.sym = g.sym; a.flags = g.flags;
  a.wait_cycles = g.wait_cycles > 0 ? g.wait_cycles : kDefaultWaitCycles;
  if (g.zsplit > 1) {  // caller-managed raw partials
    a.partial = 1; a.kchunk = g.kchunk; a.zstride = g.zstride;
    return launch(a, g.zsplit);
  }
  const int bn = a.tn;
  long long tiles = cdiv(g.M, 128) * cdiv(g.N, bn);
  if (g.sym) tiles = (tiles + 1) / 2;
  const long long rows = g.d_trans ? g.N : g.M, cols = g.d_trans ? g.M : g.N;
  int z = 1;
  const int target = g.split_target == 0 ? 152 : g.split_target;  // CTAs a split product may fill
  if (g.ws && !g.sym && target > 0 && tiles < (target * 4) / 5 && g.K >= 1024) {
    z = (int)std::min<long long>(target / tiles, g.K / 512);
    while (z > 1 && (long long)z * rows * cols > g.ws_floats) --z;
  }
  if (z > 1) {
    const int kchunk = (int)(cdiv(cdiv(g.K, z), kalign) * kalign);
    z = (int)cdiv(g.K, kchunk);
    a.partial = 1; a.kchunk = kchunk; a.D = g.ws; a.ldd = cols; a.zstride = rows * cols;
    cudaError_t e = launch(a, z);
    if (e != cudaSuccess) return e;
    const long long tot = rows * cols;
    k_reduce_epilogue<<<(unsigned)cdiv(tot, 256), 256, 0, s>>>(g.ws, z, rows * cols, (int)rows, (int)cols, g);
    note_launch();
    return cudaGetLastError();
  }
  a.partial = 0;
  a.kchunk = (int)(cdiv(g.K, kalign) * kalign);
  return launch(a, 1);
}

cudaError_t syrk_update(cudaStream_t s, int d, int K, const float* X, int ldx, float alpha, float beta,
                        kfac_precision prec, float* F, int ldf, int* flags, long long wait_cycles, const float* Xlo,
                        long long ldlo) {
  GemmDesc<float> g = {};
  g.A_lo = g.B_lo = Xlo; g.ld_alo = g.ld_blo = ldlo;
  g.M = d; g.N = d; g.K = K;
  g.A = X; g.sam = ldx; g.sak = 1;
  g.B = X; g.sbn = ldx; g.sbk = 1;
  g.D = F; g.ldd = ldf;
  g.C0 = F; g.ldc = ldf;
  g.alpha = alpha;
  g.beta = beta;
  g.zsplit = 1;
  g.sym = 1;
  g.flags = flags;
  g.wait_cycles = wait_cycles;
  return gemm_f32(g, prec, s);
}

cudaError_t ea_syrk(cudaStream_t s, int d, int n, const float* X, int ldx, float rho, kfac_precision prec, float* F,
                    int ldf, int* flags, long long wait_cycles, const float* Xlo, long long ldlo) {
  GemmDesc<float> g = {};
  g.A_lo = g.B_lo = Xlo; g.ld_alo = g.ld_blo = ldlo;
  g.M = d; g.N = d; g.K = n;
  g.A = X; g.sam = ldx; g.sak = 1;
  g.B = X; g.sbn = ldx; g.sbk = 1;
  g.D = F; g.ldd = ldf;
  g.C0 = F; g.ldc = ldf;
  g.alpha = n > 0 ? (1.0f - rho) / (float)n : 0.0f;
  g.beta = rho;
  g.zsplit = 1;
  g.sym = 1;  // upper tiles computed once, mirrored: the factor stays exactly symmetric
  g.flags = flags;
  g.wait_cycles = wait_cycles;
  if (rho == 0.0f) g.beta = 0.0f;
  return gemm_f32(g, prec, s);
}

cudaError_t tails_f32(const float* X, long long ldx, int rows, int cols, float* lo, long long ldlo, cudaStream_t s) {
  return tc::tf32_tails(X, ldx, rows, cols, lo, ldlo, s);
}

}  // namespace kfac
