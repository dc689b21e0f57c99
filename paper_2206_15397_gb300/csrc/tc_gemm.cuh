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
  long long wait_cycles;  // limit (clock cycles, > 0) of each wait for another role's progress
  int lo_a, lo_b;         // 3xTF32: the operand's tails come from global memory (set by gemm())
  int tn;                 // tile width (columns of D per CTA): a multiple of 16 up to the kernel's; 0 = widest
};

// True when A (M x K, row stride lda) and B (N x K, row stride ldb) can be read
// by TMA: 16-byte aligned bases and row strides.
bool eligible(const float* A, long long lda, const float* B, long long ldb, int M, int N, int K);

// Operand arithmetic of a launch: FP32-accurate 3xTF32 products, TF32 or
// BF16 (round to nearest) operands; FP32 accumulation in tensor memory.
enum class Mode { Fp32, Tf32, Bf16 };

// Tile width (columns of D per CTA) for N columns: the fewest tiles of the
// kernel's widest (128, or 256 for TF32 and direct-BF16 products with N > 128),
// each narrowed to the multiple of 16 that covers N evenly (k = 522 takes 5
// tiles of 112 instead of 5 of 128). Symmetric products keep square tiles.
inline int tile_n(int N, Mode mode, bool sym = false, bool bf16_direct = false) {
  const int widest = ((mode == Mode::Tf32 || bf16_direct) && N > 128) ? 256 : 128;
  if (sym || mode == Mode::Bf16 && !bf16_direct) return widest;
  const int nt = (N + widest - 1) / widest;
  const int tn = ((N + nt - 1) / nt + 15) / 16 * 16;
  return tn < widest ? tn : widest;
}

// K-columns one pipeline stage of the launch consumes.
inline int k_step(Mode mode) { return mode == Mode::Bf16 ? 64 : 32; }

// Launch one GEMM. Mode::Fp32 may take precomputed tail planes Alo / Blo
// (tf32_tails of A / B, same shape, row strides ldalo / ldblo): TMA then loads
// them beside the operands instead of the kernel forming them per tile.
cudaError_t gemm(const TcArgs& a, const float* A, long long lda, const float* B, long long ldb, int zsplit,
                 Mode mode, cudaStream_t s, const float* Alo = nullptr, long long ldalo = 0,
                 const float* Blo = nullptr, long long ldblo = 0);
// lo = the 3xTF32 tail of X (rows x cols, row strides multiples of 4 floats,
// 16-byte aligned bases).
cudaError_t tf32_tails(const float* X, long long ldx, int rows, int cols, float* lo, long long ldlo, cudaStream_t s);
// The same with A and B already BF16 in global memory (row strides lda, ldb in
// elements, multiples of 8; 16-byte aligned bases): TMA loads the BF16 tiles
// directly and tcgen05.mma.kind::f16 multiplies them; a.kchunk a multiple of 64.
cudaError_t gemm_bf16(const TcArgs& a, const void* A, long long lda, const void* B, long long ldb, int zsplit,
                      cudaStream_t s);

}  // namespace tc
}  // namespace kfac
