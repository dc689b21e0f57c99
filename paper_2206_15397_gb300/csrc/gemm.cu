// GEMM-shaped steps: dispatch and the EA SYRK.
#include "gemm.cuh"

namespace kfac {

static Round round_of(kfac_precision p) {
  return p == KFAC_PREC_BF16 ? Round::BF16 : (p == KFAC_PREC_TF32 ? Round::TF32 : Round::None);
}

cudaError_t gemm_f32(const GemmDesc<float>& g, kfac_precision prec, cudaStream_t s) {
  return gemm_simt_f32(g, round_of(prec), s);
}

cudaError_t ea_syrk(cudaStream_t s, int d, int n, const float* X, int ldx, float rho, kfac_precision prec, float* F,
                    int ldf) {
  GemmDesc<float> g = {};
  g.M = d; g.N = d; g.K = n;
  g.A = X; g.sam = ldx; g.sak = 1;
  g.B = X; g.sbn = ldx; g.sbk = 1;
  g.D = F; g.ldd = ldf;
  g.C0 = F; g.ldc = ldf;
  g.alpha = n > 0 ? (1.0f - rho) / (float)n : 0.0f;
  g.beta = rho;
  g.zsplit = 1;
  if (rho == 0.0f) g.beta = 0.0f;
  return gemm_f32(g, prec, s);
}

}  // namespace kfac
