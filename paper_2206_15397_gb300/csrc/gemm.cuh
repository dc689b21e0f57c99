// GEMM-shaped steps of the hot path and their dispatch.
#pragma once
#include <algorithm>

#include "common.cuh"

namespace kfac {

// D = alpha * rowscale * colscale * A B^T + beta * C0 in FP32 storage with the
// product arithmetic of `prec`. Dispatches to the tensor-core kernels where the
// shape and layout qualify, else to the SIMT kernel.
cudaError_t gemm_f32(const GemmDesc<float>& g, kfac_precision prec, cudaStream_t s);

// F <- rho F + (1 - rho)/n X X^T (Alg. 1 EA updates), exactly symmetric result.
// Xlo: optional precomputed 3xTF32 tails of X (row stride ldlo) for FP32 products.
cudaError_t ea_syrk(cudaStream_t s, int d, int n, const float* X, int ldx, float rho, kfac_precision prec, float* F,
                    int ldf, int* flags, long long wait_cycles = 0, const float* Xlo = nullptr, long long ldlo = 0);

// F <- beta F + alpha X X^T (exactly symmetric), X d x K with row stride ldx.
cudaError_t syrk_update(cudaStream_t s, int d, int K, const float* X, int ldx, float alpha, float beta,
                        kfac_precision prec, float* F, int ldf, int* flags, long long wait_cycles = 0,
                        const float* Xlo = nullptr, long long ldlo = 0);

// lo = the 3xTF32 tails of X (rows x cols, row strides multiples of 4 floats,
// 16-byte aligned bases), for the Xlo / A_lo / B_lo arguments above.
cudaError_t tails_f32(const float* X, long long ldx, int rows, int cols, float* lo, long long ldlo, cudaStream_t s);

}  // namespace kfac
