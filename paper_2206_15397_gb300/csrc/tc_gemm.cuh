// tcgen05 tensor-core GEMM (see tc_gemm.cu).
#pragma once
#include "common.cuh"

namespace kfac {
namespace tc {

// Epilogue and shape of one tensor-core GEMM launch. K-range per blockIdx.z is
// [z * kchunk, min(K, (z + 1) * kchunk)); kchunk must be a multiple of 32. With
// `partial`, each z writes its raw sums to D + z * zstride (no epilogue).
struct TcArgs {
  int M, N, K, kchunk;
  float alpha, beta;
  const float* rowscale;
  const float* colscale;
  const float* C0;
  long long ldc;
  int c0_trans;  // C0(m, n) = C0[n * ldc + m]
  float* D;
  long long ldd;
  int d_trans;   // D(m, n) stored at D[n * ldd + m]
  int partial;
  long long zstride;
  int sym;       // write only m <= n, plus the mirror (n, m); tiles below the diagonal exit
  int* flags;
};

// True when A (M x K, row stride lda) and B (N x K, row stride ldb) can be read
// by TMA: 16-byte aligned bases and row strides.
bool eligible(const float* A, long long lda, const float* B, long long ldb, int M, int N, int K);

// Tile width (columns of D per CTA) the launch below uses.
inline int tile_n(int N, bool split3) { return (split3 || N <= 128) ? 128 : 256; }

// Launch one GEMM: TF32 products (split3 = false) or FP32-accurate 3xTF32
// products (split3 = true), FP32 accumulation in tensor memory.
cudaError_t gemm(const TcArgs& a, const float* A, long long lda, const float* B, long long ldb, int zsplit,
                 bool split3, cudaStream_t s);

}  // namespace tc
}  // namespace kfac
