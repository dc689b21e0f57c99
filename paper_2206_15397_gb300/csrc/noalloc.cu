// Allocation-free preconditioner apply (kfac_precondition_noalloc).
//
// For callers that cannot allocate device memory when they call us: code that
// runs during CUDA graph capture, frameworks that reserve all GPU memory up
// front in their own pool, processes whose allocator is locked. The scratch
// lives in a file-scope static device array, resolved once per device with
// cudaGetSymbolAddress; nothing here calls cudaMalloc/cudaFree or any
// allocating library routine.
#include <mutex>

#include "common.cuh"
#include "gemm.cuh"

namespace {

// Shared by every call on a device; holds T (d_g x r_a), then T2 (r_g x d_a).
static __device__ __align__(256) float g_noalloc_scratch[KFAC_NOALLOC_SCRATCH_FLOATS];

constexpr int kMaxDevices = 256;
float* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Host code may not use g_noalloc_scratch as a device address (it names a
// host-side shadow); resolve the real address for the current device once.
cudaError_t scratch_for_current_device(float** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" KFAC_API kfac_status kfac_precondition_noalloc(void* stream, int d_g, int d_a, const float* J, int ldj,
                                                          const float* U_a, int ld_ua, const float* coef_a, int r_a,
                                                          const float* U_g, int ld_ug, const float* coef_g, int r_g,
                                                          float lambda, kfac_precision prec, float* S, int lds) {
  using namespace kfac;
  if (d_g < 0 || d_a < 0 || r_a < 0 || r_g < 0 || r_a > d_a || r_g > d_g) return KFAC_ERR_INVALID_ARG;
  if (!(lambda > 0.0f) || prec < KFAC_PREC_FP32 || prec > KFAC_PREC_BF16) return KFAC_ERR_INVALID_ARG;
  if ((long long)d_g * d_a == 0) return KFAC_OK;
  if (!J || ldj < d_a || !S || lds < d_a || S == J) return KFAC_ERR_INVALID_ARG;
  if (r_a > 0 && (!U_a || ld_ua < r_a || !coef_a)) return KFAC_ERR_INVALID_ARG;
  if (r_g > 0 && (!U_g || ld_ug < r_g || !coef_g)) return KFAC_ERR_INVALID_ARG;
  // T is dead once M is formed, so T2 reuses the same floats: the larger of the two must fit.
  const long long need_t = (long long)d_g * r_a, need_t2 = (long long)r_g * d_a;
  if (need_t > (long long)KFAC_NOALLOC_SCRATCH_FLOATS || need_t2 > (long long)KFAC_NOALLOC_SCRATCH_FLOATS)
    return KFAC_ERR_TOO_LARGE;

  float* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return KFAC_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* T = scratch;   // d_g x r_a
  float* T2 = scratch;  // r_g x d_a, written only after the M product has consumed T (stream order)
  const float inv_lam = 1.0f / lambda;
  if (r_a > 0) {  // T = J U_a diag(c_a)
    GemmDesc<float> g = {};
    g.M = d_g; g.N = r_a; g.K = d_a;
    g.A = J; g.sam = ldj; g.sak = 1;
    g.B = U_a; g.sbn = 1; g.sbk = ld_ua;
    g.D = T; g.ldd = r_a;
    g.alpha = 1.0f; g.colscale = coef_a; g.zsplit = 1;
    if (gemm_f32(g, prec, s) != cudaSuccess) return KFAC_ERR_CUDA;
  }
  {  // M = T U_a^T + J / lambda, staged in S
    GemmDesc<float> g = {};
    g.M = d_g; g.N = d_a; g.K = r_a;
    g.A = T; g.sam = r_a > 0 ? r_a : 1; g.sak = 1;
    g.B = U_a; g.sbn = ld_ua; g.sbk = 1;
    g.D = S; g.ldd = lds;
    g.alpha = 1.0f; g.beta = inv_lam; g.C0 = J; g.ldc = ldj; g.zsplit = 1;
    if (gemm_f32(g, prec, s) != cudaSuccess) return KFAC_ERR_CUDA;
  }
  if (r_g > 0) {
    {  // T2 = diag(c_g) U_g^T M
      GemmDesc<float> g = {};
      g.M = r_g; g.N = d_a; g.K = d_g;
      g.A = U_g; g.sam = 1; g.sak = ld_ug;
      g.B = S; g.sbn = 1; g.sbk = lds;
      g.D = T2; g.ldd = d_a;
      g.alpha = 1.0f; g.rowscale = coef_g; g.zsplit = 1;
      if (gemm_f32(g, prec, s) != cudaSuccess) return KFAC_ERR_CUDA;
    }
    {  // S = U_g T2 + M / lambda, in place (each element is read, then written, by one thread)
      GemmDesc<float> g = {};
      g.M = d_g; g.N = d_a; g.K = r_g;
      g.A = U_g; g.sam = ld_ug; g.sak = 1;
      g.B = T2; g.sbn = 1; g.sbk = d_a;
      g.D = S; g.ldd = lds;
      g.alpha = 1.0f; g.beta = inv_lam; g.C0 = S; g.ldc = lds; g.zsplit = 1;
      if (gemm_f32(g, prec, s) != cudaSuccess) return KFAC_ERR_CUDA;
    }
  } else {  // S = M / lambda
    GemmDesc<float> g = {};
    g.M = d_g; g.N = d_a; g.K = 0;
    g.A = U_g; g.sam = 1; g.sak = 1;
    g.B = J; g.sbn = 1; g.sbk = 1;
    g.D = S; g.ldd = lds;
    g.alpha = 1.0f; g.beta = inv_lam; g.C0 = S; g.ldc = lds; g.zsplit = 1;
    if (gemm_f32(g, prec, s) != cudaSuccess) return KFAC_ERR_CUDA;
  }
  return KFAC_OK;
}
