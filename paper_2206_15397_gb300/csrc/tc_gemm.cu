// Tensor-core GEMM for sm_100-family (tcgen05 + TMA + TMEM), FP32 storage.
//
//   D[m, n] = alpha * rowscale[m] * colscale[n] * sum_k A[m, k] B[n, k] + beta * C0(m, n)
//
// A (M x K) and B (N x K) are row-major with K contiguous ("K-major"). One CTA
// computes a 128 x BN tile:
//   * warp 0 / lane 0 streams A and B tiles of 32 FP32 columns (128 bytes = one
//     128B-swizzle row) with cp.async.bulk.tensor into a ring of shared-memory
//     stages, each guarded by a "full" mbarrier (transaction bytes);
//   * warp 1 / lane 0 issues tcgen05.mma.kind::tf32 (M = 128, N = BN, K = 8 per
//     instruction) into TMEM and hands each stage back with tcgen05.commit ->
//     "empty";
//   * the accumulator is read with tcgen05.ld (warp w reads TMEM lanes
//     32*(w%4)..+31), the epilogue applied and D stored. Row-major D / C0 go
//     through a per-warp shared-memory tile so global accesses are coalesced;
//     transposed D / C0 (D[n][m]) are coalesced directly since TMEM lanes are
//     consecutive rows.
// Two kernels:
//   k_tc_gemm   TF32 products, one accumulator over the CTA's whole K range
//               (all 8 warps share the epilogue).
//   k_tc_gemm3  FP32-accurate products (3xTF32): the staged FP32 tile is the
//               head operand as it stands (the tensor core reads it truncated
//               to TF32); warps 2-7 write each value's tail, the rest below
//               that truncation rounded to TF32, and fence the writes for the
//               async proxy; the issuer
//               puts hi*hi into one accumulator and hi*lo + lo*hi into
//               another. The tensor core's FP32 accumulation rounds toward
//               zero, which over a long K loop drifts every sum low (measured
//               about -5e-6 relative over K = 512 with one accumulator), so
//               every two stages (K = 64) accumulate into a fresh TMEM pair,
//               double buffered, and warps 4-7, between splitting the next
//               stages, add every finished pair into FP32 registers with
//               round-to-nearest. The remaining bias is that of eight K-steps
//               (measured -2e-7 relative, independent of K; -9e-8 with one
//               stage per pair, which drained twice as often and ran 6%
//               slower).
//   k_tc_gemm16 BF16 operands (the reduced-precision path): TMA stages FP32
//               tiles of 64 K-columns (two 32-column boxes per operand) in a
//               ring of its own; warps 2-7 round them to BF16 (round to nearest)
//               into a second ring of 128-byte-swizzled K-major tiles and hand
//               the FP32 stage straight back to TMA; warp 1 issues
//               tcgen05.mma.kind::f16 (BF16 x BF16, K = 16 per instruction,
//               FP32 accumulator in TMEM).
// Every mbarrier wait is bounded by a clock deadline; on expiry the kernel
// raises KFAC_FLAG_TIMEOUT, drains what it issued and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace kfac {
namespace tc {
namespace {

constexpr int BM = 128;
constexpr int BK = 32;  // FP32 columns per stage (128 bytes)
constexpr int THREADS = 256;
// Limit of the waits for this CTA's own work in flight (its TMA copies landing,
// its MMAs completing): those always finish, so the limit is long (~2 s at
// 2 GHz) and independent of TcArgs::wait_cycles, which bounds the waits for
// another role's progress. A CTA whose peer wait gave up therefore still
// exits only after its copies and MMAs have completed.
constexpr long long kDrainCycles = 4000000000LL;
constexpr int BN3 = 128;            // tile width of the FP32-accurate kernel
constexpr int kSplitThreads = 192;  // warps 2-7 split the staged tiles (3xTF32)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `bar` with the given parity to complete, or give up
// after `limit` clock cycles (raising the timeout flag). Returns true on
// completion.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* flags, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) {
      raise_flag(flags, KFAC_FLAG_TIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// As tmem_ld32 without the wait: the registers are valid after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_k128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;            // leading-dimension offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride-dimension offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;            // descriptor format constant
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Instruction descriptor of kind::f16 with BF16 A and B, F32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Two FP32 values rounded to nearest BF16, packed low = a, high = b.
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}

// x rounded to nearest TF32 (exactly representable in TF32). Rounding (not
// truncation) keeps the tail |x - hi| <= 2^-11 |x| and unbiased: truncated heads
// leave tails of one sign that the tensor core truncates again, biasing every
// product low by ~1e-6, which chained products accumulate.

template <int BN>
struct Cfg {
  static constexpr int A_BYTES = BM * BK * 4;
  static constexpr int B_BYTES = BN * BK * 4;
  static constexpr int RAW = A_BYTES + B_BYTES;
  static constexpr int STAGE = RAW;
  static constexpr int STAGES = (196608 / STAGE) < 8 ? (196608 / STAGE) : 8;
  static constexpr int BAR_BYTES = 8 * (2 * STAGES + 1) + 16;
  static constexpr int SMEM = 1024 + STAGES * STAGE + BAR_BYTES;
};

// FP32-accurate kernel: stages carry the raw tile and the tail tile.
struct Cfg3 {
  static constexpr int A_BYTES = BM * BK * 4;
  static constexpr int B_BYTES = BN3 * BK * 4;
  static constexpr int RAW = A_BYTES + B_BYTES;
  static constexpr int STAGE = 2 * RAW;
  static constexpr int STAGES = 196608 / STAGE;
  static constexpr int BAR_BYTES = 8 * (3 * STAGES + 5) + 16;
  static constexpr int SMEM = 1024 + STAGES * STAGE + BAR_BYTES;
  static constexpr int TMEM_COLS = 4 * BN3;  // main[2], small[2]
};

// BF16 kernel: FP32 stages of 64 K-columns (2 boxes per operand) and BF16
// stages of the same K-range (one 128-byte row per matrix row).
constexpr int BN16 = 128;
constexpr int BK16 = 64;
constexpr int kConvThreads = 192;  // warps 2-7
struct Cfg16 {
  static constexpr int A_RAW = BM * BK16 * 4;
  static constexpr int B_RAW = BN16 * BK16 * 4;
  static constexpr int RAW = A_RAW + B_RAW;
  static constexpr int A_H = BM * BK16 * 2;
  static constexpr int B_H = BN16 * BK16 * 2;
  static constexpr int HALF = A_H + B_H;
  static constexpr int RAW_STAGES = 2, H_STAGES = 2;
  static constexpr int BAR_BYTES = 8 * (2 * RAW_STAGES + 2 * H_STAGES + 1) + 16;
  static constexpr int SMEM = 1024 + RAW_STAGES * RAW + H_STAGES * HALF + BAR_BYTES;
};

// Epilogue of 32 consecutive columns [nb, nb + 32) of row m held by this lane
// (v[j] = raw sum for column nb + j): scaling, beta * C0, store (row-major via
// the warp's staging tile, or transposed), the symmetric mirror.
__device__ __forceinline__ void store_chunk(const TcArgs& p, float (&v)[32], int m, int mrow0, int nb, int lane,
                                            float rs, float* stage_tile, float* Dz, int nend) {
  if (!p.partial) {
    float cin[32];
    if (p.beta != 0.0f && p.C0) {
      if (p.c0_trans) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = nb + j;
          cin[j] = (m < p.M && n < nend) ? p.C0[(long long)n * p.ldc + m] : 0.0f;
        }
      } else {  // rows of C0 through the staging tile: all 32 row loads in flight, then the stores
        float rowv[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int mr = mrow0 + r, n = nb + lane;
          rowv[r] = (mr < p.M && n < nend) ? __ldg(p.C0 + (long long)mr * p.ldc + n) : 0.0f;
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 32; ++r) stage_tile[r * 33 + lane] = rowv[r];
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 32; ++j) cin[j] = stage_tile[lane * 33 + j];
      }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int n = nb + j;
      float x = v[j] * p.alpha * rs;
      if (p.colscale && n < nend) x *= p.colscale[n];
      if (p.beta != 0.0f && p.C0) x = fmaf(p.beta, cin[j], x);
      v[j] = x;
    }
  }
  if (p.d_trans) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int n = nb + j;
      if (m < p.M && n < nend) Dz[(long long)n * p.ldd + m] = v[j];
    }
  } else {
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; ++j) stage_tile[lane * 33 + j] = v[j];
    __syncwarp();
    for (int r = 0; r < 32; ++r) {
      const int mr = mrow0 + r, n = nb + lane;
      if (mr < p.M && n < nend && (!p.sym || mr <= n)) Dz[(long long)mr * p.ldd + n] = stage_tile[r * 33 + lane];
    }
    if (p.sym && !p.partial) {  // mirror: D[n][m] for m < n (raw split-K partials keep the upper triangle only)
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = nb + j;
        if (m < p.M && n < nend && m < n) Dz[(long long)n * p.ldd + m] = v[j];
      }
    }
  }
}

// BF16D: A and B are BF16 in global memory (64 K-columns = 128 bytes per
// stage row, tcgen05.mma.kind::f16 with K = 16); otherwise FP32 read as TF32
// (32 K-columns per stage row, kind::tf32 with K = 8). The shared-memory tiles
// have the same shape and swizzle either way.
template <int BN, bool BF16D = false>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs p) {
  using C = Cfg<BN>;
  constexpr int BK = BF16D ? 64 : 32;  // K elements per stage (128-byte rows)
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * C::STAGES + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * C::STAGES;
  const uint32_t accb = empty0 + 8 * C::STAGES;
  __shared__ int s_abort;  // a wait of this CTA gave up: the accumulator is not a result

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tn = p.tn;  // this launch's tile width: a multiple of 16, at most BN
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * tn;
  const int nend = min(p.N, n0 + tn);
  if (p.sym && m0 > n0 + tn - 1) return;  // whole tile below the diagonal (uniform exit, nothing started)
  const int kb0 = blockIdx.z * p.kchunk;
  const int ke = min(p.K, kb0 + p.kchunk);
  const int nk = ke > kb0 ? (ke - kb0 + BK - 1) / BK : 0;
  const uint32_t stage_tx = (uint32_t)(C::A_BYTES + tn * (C::B_BYTES / BN));

  if (tid == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accb, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer --------------------------------------------------------
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % C::STAGES;
      const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
      if (kb >= C::STAGES && !mbar_wait(empty0 + 8 * s, ph ^ 1u, p.flags, p.wait_cycles)) { s_abort = 1; break; }
      const uint32_t st = smem_u32(smem + s * C::STAGE);
      mbar_expect_tx(full0 + 8 * s, stage_tx);
      tma_load_2d(st, &tmA, kb0 + kb * BK, m0, full0 + 8 * s);
      tma_load_2d(st + C::A_BYTES, &tmB, kb0 + kb * BK, n0, full0 + 8 * s);
      ++issued;
    }
    // Drain: every issued copy has landed before this CTA may exit (the MMA
    // issuer consumes them in the normal path; this matters after a timeout).
    for (int kb = (issued > C::STAGES ? issued - C::STAGES : 0); kb < issued; ++kb)
      mbar_wait(full0 + 8 * (kb % C::STAGES), (uint32_t)(kb / C::STAGES) & 1u, p.flags, kDrainCycles);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----------------------------------------------------------
    const uint32_t idesc = BF16D ? idesc_bf16(BM, tn) : idesc_tf32(BM, tn);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % C::STAGES;
      const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
      if (!mbar_wait(full0 + 8 * s, ph, p.flags, p.wait_cycles)) { s_abort = 1; break; }
      tc_fence_after();
      const uint32_t st = smem_u32(smem + s * C::STAGE);
      const uint64_t ad = sdesc_k128(st), bd = sdesc_k128(st + C::A_BYTES);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {  // 32 bytes of K per instruction: 8 TF32 or 16 BF16
        const uint64_t off = (uint64_t)(kk * 2);  // 32 bytes >> 4
        if (BF16D) mma_bf16(taddr, ad + off, bd + off, idesc, (kb | kk) ? 1u : 0u);
        else mma_tf32(taddr, ad + off, bd + off, idesc, (kb | kk) ? 1u : 0u);
      }
      mma_commit(empty0 + 8 * s);  // stage reusable once these MMAs completed
    }
    mma_commit(accb);  // accumulator ready (also completes when nothing was issued)
  }
  __syncthreads();  // s_abort is final

  // ---- epilogue ----------------------------------------------------------------
  const bool acc_ok = mbar_wait(accb, 0, p.flags, kDrainCycles) && !s_abort;  // every issued MMA has completed
  tc_fence_after();
  float* stage_tile = reinterpret_cast<float*>(smem) + warp * (32 * 33);  // per-warp 32 x 33 staging
  float* const Dz = p.D + (p.partial ? (long long)blockIdx.z * p.zstride : 0LL);  // split-K slice
  const int q = warp & 3;
  const int m = m0 + 32 * q + lane;
  const int cbeg = (warp < 4) ? 0 : BN / 2;
  const float rs = (p.rowscale && m < p.M) ? p.rowscale[m] : 1.0f;
  for (int c0 = cbeg; c0 < cbeg + BN / 2; c0 += 32) {
    const int nb = n0 + c0;
    if (nb >= nend) break;  // uniform across the warp
    float v[32];
    if (nk > 0 && acc_ok) {
      tmem_ld32(taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = 0.0f;
    }
    store_chunk(p, v, m, m0 + 32 * q, nb, lane, rs, stage_tile, Dz, nend);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(BN) : "memory");
  }
}

// Warp-uniform bounded wait: lane 0 polls, the outcome is broadcast.
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, int* flags, int lane, long long limit) {
  int ok = 1;
  if (lane == 0) ok = mbar_wait(bar, parity, flags, limit) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gemm3(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmAlo, const __grid_constant__ CUtensorMap tmBlo, TcArgs p) {
  using C = Cfg3;
  // Operands whose tails come precomputed from global memory (p.lo_a / p.lo_b)
  // are loaded by TMA beside the raw tile; the split warps form the others'.
  // With both precomputed no split runs: the MMA issuer takes a stage as soon
  // as its copies have landed.
  const bool need_split = !(p.lo_a && p.lo_b);
  const int b_bytes = p.tn * (C::B_BYTES / BN3);  // the B tile's rows that TMA fills
  const uint32_t stage_tx = (uint32_t)(C::A_BYTES + b_bytes + (p.lo_a ? C::A_BYTES : 0) + (p.lo_b ? b_bytes : 0));
  const int split_e0 = p.lo_a ? C::A_BYTES / 16 : 0;             // float4 range of the stage to split
  const int split_e1 = p.lo_b ? C::A_BYTES / 16 : (C::A_BYTES + b_bytes) / 16;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * C::STAGES + 5);
  const uint32_t full0 = smem_u32(bars), split0 = full0 + 8 * C::STAGES, empty0 = split0 + 8 * C::STAGES;
  const uint32_t tfull0 = empty0 + 8 * C::STAGES, tempty0 = tfull0 + 16, accb = tempty0 + 16;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tn = p.tn;  // this launch's tile width: a multiple of 16, at most BN3
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * tn;
  const int nend = min(p.N, n0 + tn);
  if (p.sym && m0 > n0 + tn - 1) return;  // whole tile below the diagonal (uniform exit, nothing started)
  const int kb0 = blockIdx.z * p.kchunk;
  const int ke = min(p.K, kb0 + p.kchunk);
  const int nk = ke > kb0 ? (ke - kb0 + BK - 1) / BK : 0;

  if (tid == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(split0 + 8 * s, kSplitThreads);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, 4);  // one arrival per drain warp
    }
    mbar_init(accb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *tmem_slot;

  float acc[BN3];  // warps 4-7: this lane's row of the tile, FP32 round-to-nearest sums
  bool drained = true;
  if (warp == 0 && lane == 0) {
    // ---- TMA producer --------------------------------------------------------
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % C::STAGES;
      const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
      if (kb >= C::STAGES && !mbar_wait(empty0 + 8 * s, ph ^ 1u, p.flags, p.wait_cycles)) break;
      const uint32_t st = smem_u32(smem + s * C::STAGE);
      mbar_expect_tx(full0 + 8 * s, stage_tx);
      tma_load_2d(st, &tmA, kb0 + kb * BK, m0, full0 + 8 * s);
      tma_load_2d(st + C::A_BYTES, &tmB, kb0 + kb * BK, n0, full0 + 8 * s);
      if (p.lo_a) tma_load_2d(st + C::RAW, &tmAlo, kb0 + kb * BK, m0, full0 + 8 * s);
      if (p.lo_b) tma_load_2d(st + C::RAW + C::A_BYTES, &tmBlo, kb0 + kb * BK, n0, full0 + 8 * s);
      ++issued;
    }
    for (int kb = (issued > C::STAGES ? issued - C::STAGES : 0); kb < issued; ++kb)
      mbar_wait(full0 + 8 * (kb % C::STAGES), (uint32_t)(kb / C::STAGES) & 1u, p.flags, kDrainCycles);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: stages 2m, 2m+1 -> TMEM pair m & 1 ------------------------
    const uint32_t ready0 = need_split ? split0 : full0;
    const uint32_t idesc = idesc_tf32(BM, tn);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % C::STAGES, m = kb >> 1, b = m & 1;
      const bool first = (kb & 1) == 0, last = (kb & 1) == 1 || kb == nk - 1;
      const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
      if (first && m >= 2 && !mbar_wait(tempty0 + 8 * b, (uint32_t)((m >> 1) - 1) & 1u, p.flags, p.wait_cycles)) break;
      if (!mbar_wait(ready0 + 8 * s, ph, p.flags, p.wait_cycles)) break;
      tc_fence_after();
      const uint32_t st = smem_u32(smem + s * C::STAGE);
      const uint64_t ad = sdesc_k128(st), bd = sdesc_k128(st + C::A_BYTES);
      const uint64_t adl = sdesc_k128(st + C::RAW), bdl = sdesc_k128(st + C::RAW + C::A_BYTES);
      const uint32_t tmain = taddr + (uint32_t)(b * BN3), tsmall = taddr + (uint32_t)(2 * BN3 + b * BN3);  // pair b
#pragma unroll
      for (int kk = 0; kk < BK / 8; ++kk) {
        const uint64_t off = (uint64_t)(kk * 2);
        const uint32_t acc0 = (kk || !first) ? 1u : 0u;
        mma_tf32(tmain, ad + off, bd + off, idesc, acc0);
        mma_tf32(tsmall, ad + off, bdl + off, idesc, acc0);
        mma_tf32(tsmall, adl + off, bd + off, idesc, 1u);
      }
      mma_commit(empty0 + 8 * s);          // stage reusable once these MMAs completed
      if (last) mma_commit(tfull0 + 8 * b);  // pair b holds the sums of stages 2m, 2m+1
    }
    mma_commit(accb);  // every issued MMA has completed (also when nothing was issued)
  } else if (warp >= 2) {
    // ---- warps 2-7: 3xTF32 split of stage kb; warps 4-7 then drain pairs ------
    // hi is the staged FP32 value itself, which the tensor core reads truncated
    // to TF32; lo = RN_tf32(x - trunc(x)) goes to the second half of the stage,
    // so hi*hi + hi*lo + lo*hi carries x*y to ~2^-21 relative, unbiased. All
    // waits here are warp-uniform so the warp stays converged for tcgen05.ld.
    const int t = tid - 64;
    const bool drainer = warp >= 4;
    const uint32_t lrow = (uint32_t)(32 * (warp & 3)) << 16;
    if (drainer) {
#pragma unroll
      for (int j = 0; j < BN3; ++j) acc[j] = 0.0f;
    }
    for (int kb = 0; kb <= nk; ++kb) {
      if (kb < nk && need_split) {
        const int s = kb % C::STAGES;
        const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
        if (!mbar_wait_warp(full0 + 8 * s, ph, p.flags, lane, p.wait_cycles)) { drained = false; break; }
        const float4* raw = reinterpret_cast<const float4*>(smem + s * C::STAGE);
        float4* lo = reinterpret_cast<float4*>(smem + s * C::STAGE + C::RAW);
#pragma unroll 2
        for (int e = split_e0 + t; e < split_e1; e += kSplitThreads) {
          const float4 x = raw[e];  // read as hi by the tensor core (its TF32 truncation)
          lo[e] = make_float4(tf32_tail(x.x), tf32_tail(x.y), tf32_tail(x.z), tf32_tail(x.w));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(split0 + 8 * s);
      }
      if (drainer && kb >= 1 && (((kb - 1) & 1) == 1 || kb == nk)) {  // pair of stages ending at kb - 1
        const int m = (kb - 1) >> 1, b = m & 1;
        if (!mbar_wait_warp(tfull0 + 8 * b, (uint32_t)(m >> 1) & 1u, p.flags, lane, p.wait_cycles)) { drained = false; break; }
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < BN3 / 32; ++c) {
          if (32 * c >= tn) break;  // columns this tile's MMAs never wrote (warp-uniform)
          uint32_t v[32], w[32];
          tmem_ld32_async(taddr + lrow + (uint32_t)(b * BN3 + 32 * c), v);
          tmem_ld32_async(taddr + lrow + (uint32_t)(2 * BN3 + b * BN3 + 32 * c), w);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 32; ++j) acc[32 * c + j] += __uint_as_float(v[j]) + __uint_as_float(w[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty0 + 8 * b);
      }
    }
  }
  __syncwarp();

  // ---- epilogue (warps 4-7, from the register sums) ---------------------------
  const bool acc_ok = mbar_wait_warp(accb, 0, p.flags, lane, kDrainCycles);  // every issued MMA has completed
  tc_fence_after();
  if (warp >= 4) {
    float* stage_tile = reinterpret_cast<float*>(smem) + warp * (32 * 33);
    float* const Dz = p.D + (p.partial ? (long long)blockIdx.z * p.zstride : 0LL);
    const int q = warp & 3;
    const int m = m0 + 32 * q + lane;
    const float rs = (p.rowscale && m < p.M) ? p.rowscale[m] : 1.0f;
    const bool ok = acc_ok && drained;
#pragma unroll
    for (int c = 0; c < BN3 / 32; ++c) {
      const int nb = n0 + 32 * c;
      if (nb < nend) {  // uniform across the warp
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = ok ? acc[32 * c + j] : 0.0f;
        store_chunk(p, v, m, m0 + 32 * q, nb, lane, rs, stage_tile, Dz, nend);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(C::TMEM_COLS)
                 : "memory");
  }
}

__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gemm16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs p) {
  using C = Cfg16;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* raw0 = smem;                                 // FP32 stages
  uint8_t* half0 = smem + C::RAW_STAGES * C::RAW;       // BF16 stages
  uint64_t* bars = reinterpret_cast<uint64_t*>(half0 + C::H_STAGES * C::HALF);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * C::RAW_STAGES + 2 * C::H_STAGES + 1);
  const uint32_t rfull0 = smem_u32(bars), rempty0 = rfull0 + 8 * C::RAW_STAGES;
  const uint32_t hfull0 = rempty0 + 8 * C::RAW_STAGES, hempty0 = hfull0 + 8 * C::H_STAGES;
  const uint32_t accb = hempty0 + 8 * C::H_STAGES;
  __shared__ int s_abort;  // a wait of this CTA gave up: the accumulator is not a result

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN16;
  if (p.sym && m0 > n0 + BN16 - 1) return;  // whole tile below the diagonal (uniform exit, nothing started)
  const int kb0 = blockIdx.z * p.kchunk;
  const int ke = min(p.K, kb0 + p.kchunk);
  const int nk = ke > kb0 ? (ke - kb0 + BK16 - 1) / BK16 : 0;

  if (tid == 0) {
    for (int s = 0; s < C::RAW_STAGES; ++s) {
      mbar_init(rfull0 + 8 * s, 1);
      mbar_init(rempty0 + 8 * s, kConvThreads);
    }
    for (int h = 0; h < C::H_STAGES; ++h) {
      mbar_init(hfull0 + 8 * h, kConvThreads);
      mbar_init(hempty0 + 8 * h, 1);
    }
    mbar_init(accb, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(BN16)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: 64 K-columns = two 32-column boxes per operand --------
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % C::RAW_STAGES;
      const uint32_t ph = (uint32_t)(kb / C::RAW_STAGES) & 1u;
      if (kb >= C::RAW_STAGES && !mbar_wait(rempty0 + 8 * s, ph ^ 1u, p.flags, p.wait_cycles)) { s_abort = 1; break; }
      const uint32_t st = smem_u32(raw0 + s * C::RAW);
      const int kx = kb0 + kb * BK16;
      mbar_expect_tx(rfull0 + 8 * s, C::RAW);
      tma_load_2d(st, &tmA, kx, m0, rfull0 + 8 * s);
      tma_load_2d(st + C::A_RAW / 2, &tmA, kx + 32, m0, rfull0 + 8 * s);
      tma_load_2d(st + C::A_RAW, &tmB, kx, n0, rfull0 + 8 * s);
      tma_load_2d(st + C::A_RAW + C::B_RAW / 2, &tmB, kx + 32, n0, rfull0 + 8 * s);
      ++issued;
    }
    for (int kb = (issued > C::RAW_STAGES ? issued - C::RAW_STAGES : 0); kb < issued; ++kb)
      mbar_wait(rfull0 + 8 * (kb % C::RAW_STAGES), (uint32_t)(kb / C::RAW_STAGES) & 1u, p.flags, kDrainCycles);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: 4 x (K = 16) per BF16 stage -----------------------------
    constexpr uint32_t idesc = idesc_bf16(BM, BN16);
    for (int kb = 0; kb < nk; ++kb) {
      const int h = kb % C::H_STAGES;
      const uint32_t ph = (uint32_t)(kb / C::H_STAGES) & 1u;
      if (!mbar_wait(hfull0 + 8 * h, ph, p.flags, p.wait_cycles)) { s_abort = 1; break; }
      tc_fence_after();
      const uint32_t hb = smem_u32(half0 + h * C::HALF);
      const uint64_t ad = sdesc_k128(hb), bd = sdesc_k128(hb + C::A_H);
#pragma unroll
      for (int kk = 0; kk < BK16 / 16; ++kk) {  // K = 16 BF16 = 32 bytes per instruction
        const uint64_t off = (uint64_t)(kk * 2);
        mma_bf16(taddr, ad + off, bd + off, idesc, (kb | kk) ? 1u : 0u);
      }
      mma_commit(hempty0 + 8 * h);  // BF16 stage reusable once these MMAs completed
    }
    mma_commit(accb);
  } else if (warp >= 2) {
    // ---- converters: FP32 (TMA 128B swizzle) -> BF16 (128B swizzle) ----------
    // An FP32 box row r holds 32 values in 8 chunks of 16 bytes, chunk c at
    // physical chunk c ^ (r % 8); a BF16 row holds the 64 values of both boxes
    // in 8 chunks of 8 values, chunk j at physical chunk j ^ (r % 8).
    const int t = tid - 64;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % C::RAW_STAGES, h = kb % C::H_STAGES;
      if (!mbar_wait_warp(rfull0 + 8 * s, (uint32_t)(kb / C::RAW_STAGES) & 1u, p.flags, lane, p.wait_cycles)) { s_abort = 1; break; }
      if (kb >= C::H_STAGES &&
          !mbar_wait_warp(hempty0 + 8 * h, ((uint32_t)(kb / C::H_STAGES) & 1u) ^ 1u, p.flags, lane, p.wait_cycles))
        { s_abort = 1; break; }
      const uint8_t* rs = raw0 + s * C::RAW;
      uint8_t* hs = half0 + h * C::HALF;
      for (int q = t; q < (BM + BN16) * 8; q += kConvThreads) {
        const int row = q >> 3, j = q & 7;
        const bool isB = row >= BM;
        const int r = isB ? row - BM : row;
        const uint8_t* box = rs + (isB ? C::A_RAW : 0) + (j >> 2) * (isB ? C::B_RAW / 2 : C::A_RAW / 2) + r * 128;
        const int c0 = 2 * (j & 3), sw = r & 7;
        const float4 x0 = *reinterpret_cast<const float4*>(box + ((c0 ^ sw) << 4));
        const float4 x1 = *reinterpret_cast<const float4*>(box + (((c0 + 1) ^ sw) << 4));
        uint4 o;
        o.x = pack_bf16x2(x0.x, x0.y);
        o.y = pack_bf16x2(x0.z, x0.w);
        o.z = pack_bf16x2(x1.x, x1.y);
        o.w = pack_bf16x2(x1.z, x1.w);
        *reinterpret_cast<uint4*>(hs + (isB ? C::A_H : 0) + r * 128 + ((j ^ sw) << 4)) = o;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(hfull0 + 8 * h);
      mbar_arrive(rempty0 + 8 * s);
    }
  }
  __syncthreads();  // s_abort is final

  // ---- epilogue (all 8 warps, as the TF32 kernel) --------------------------------
  const bool acc_ok = mbar_wait(accb, 0, p.flags, kDrainCycles) && !s_abort;  // every issued MMA has completed
  tc_fence_after();
  float* stage_tile = reinterpret_cast<float*>(smem) + warp * (32 * 33);
  float* const Dz = p.D + (p.partial ? (long long)blockIdx.z * p.zstride : 0LL);
  const int q = warp & 3;
  const int m = m0 + 32 * q + lane;
  const int cbeg = (warp < 4) ? 0 : BN16 / 2;
  const float rs = (p.rowscale && m < p.M) ? p.rowscale[m] : 1.0f;
  for (int c0 = cbeg; c0 < cbeg + BN16 / 2; c0 += 32) {
    const int nb = n0 + c0;
    if (nb >= p.N) break;
    float v[32];
    if (nk > 0 && acc_ok) {
      tmem_ld32(taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = 0.0f;
    }
    store_chunk(p, v, m, m0 + 32 * q, nb, lane, rs, stage_tile, Dz, p.N);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(BN16) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      cudaGetLastError();
  }
  return fn;
}

// 2-D map of a row-major FP32 matrix (rows x cols, row stride ld) read in
// boxes of 32 columns x box_rows rows with the 128-byte swizzle.
bool make_map(CUtensorMap* map, const void* ptr, int rows, int cols, long long ld, int box_rows, bool bf16 = false) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int esz = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * esz};
  cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};  // 128-byte rows
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// `bn` is the kernel's largest tile width; the launch uses a.tn (set here to
// bn unless the caller chose a narrower multiple of 16 that fits N better).
template <typename Kern>
cudaError_t launch_kernel(Kern kern, int smem, int bn, const TcArgs& a0, const void* A, long long lda,
                          const void* B, long long ldb, int zsplit, cudaStream_t s, bool bf16 = false) {
  {
    cudaError_t e = set_kernel_attrs_once(reinterpret_cast<const void*>(kern), smem, false);
    if (e != cudaSuccess) return e;
  }
  TcArgs a = a0;
  if (a.tn <= 0 || a.tn > bn || (a.tn & 15)) a.tn = bn;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, a.M, a.K, lda, BM, bf16) || !make_map(&mb, B, a.N, a.K, ldb, a.tn, bf16))
    return cudaErrorInvalidValue;
  dim3 grid((a.N + a.tn - 1) / a.tn, (a.M + BM - 1) / BM, zsplit);
  kern<<<grid, THREADS, smem, s>>>(ma, mb, a);
  note_launch();
  return cudaGetLastError();
}

// lo[r][c] = tail of X[r][c] below its TF32 truncation (as the 3xTF32 kernel
// forms in shared memory), four columns per thread.
__global__ void k_tf32_tails(const float* __restrict__ X, long long ldx, int rows, int cols, int cols4,
                             float* __restrict__ lo, long long ldlo) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)rows * cols4) return;
  const int r = (int)(idx / cols4), c = (int)(idx % cols4) * 4;
  const float* x = X + (long long)r * ldx + c;
  float* y = lo + (long long)r * ldlo + c;
  if (c + 4 <= cols) {
    const float4 v = *reinterpret_cast<const float4*>(x);
    *reinterpret_cast<float4*>(y) = make_float4(tf32_tail(v.x), tf32_tail(v.y), tf32_tail(v.z), tf32_tail(v.w));
  } else {  // ragged row end: only the row's own columns are read
    for (int j = 0; c + j < cols; ++j) y[j] = tf32_tail(x[j]);
  }
}

}  // namespace

cudaError_t tf32_tails(const float* X, long long ldx, int rows, int cols, float* lo, long long ldlo, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  if ((ldx & 3) || (ldlo & 3) || ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(lo)) & 15u))
    return cudaErrorInvalidValue;
  const int cols4 = (cols + 3) / 4;
  const long long n = (long long)rows * cols4;
  k_tf32_tails<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(X, ldx, rows, cols, cols4, lo, ldlo);
  note_launch();
  return cudaGetLastError();
}

cudaError_t gemm_bf16(const TcArgs& a, const void* A, long long lda, const void* B, long long ldb, int zsplit,
                      cudaStream_t s) {
  if (a.N > 128) return launch_kernel(k_tc_gemm<256, true>, Cfg<256>::SMEM, 256, a, A, lda, B, ldb, zsplit, s, true);
  return launch_kernel(k_tc_gemm<128, true>, Cfg<128>::SMEM, 128, a, A, lda, B, ldb, zsplit, s, true);
}

bool eligible(const float* A, long long lda, const float* B, long long ldb, int M, int N, int K) {
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  return M > 0 && N > 0 && K > 0 && al16(A) && al16(B) && (lda % 4) == 0 && (ldb % 4) == 0 && lda >= K && ldb >= K &&
         encode_fn() != nullptr;
}

cudaError_t gemm(const TcArgs& a0, const float* A, long long lda, const float* B, long long ldb, int zsplit,
                 Mode mode, cudaStream_t s, const float* Alo, long long ldalo, const float* Blo, long long ldblo) {
  if (mode == Mode::Fp32) {
    {
      cudaError_t e = set_kernel_attrs_once(reinterpret_cast<const void*>(k_tc_gemm3), Cfg3::SMEM, false);
      if (e != cudaSuccess) return e;
    }
    TcArgs a = a0;
    a.lo_a = Alo != nullptr;
    a.lo_b = Blo != nullptr;
    if (a.tn <= 0 || a.tn > BN3 || (a.tn & 15)) a.tn = BN3;
    // Tail planes share their operand's shape; an absent one gets its
    // operand's map (never read).
    CUtensorMap ma, mb, mal, mbl;
    if (!make_map(&ma, A, a.M, a.K, lda, BM) || !make_map(&mb, B, a.N, a.K, ldb, a.tn) ||
        !make_map(&mal, Alo ? Alo : A, a.M, a.K, Alo ? ldalo : lda, BM) ||
        !make_map(&mbl, Blo ? Blo : B, a.N, a.K, Blo ? ldblo : ldb, a.tn))
      return cudaErrorInvalidValue;
    dim3 grid((a.N + a.tn - 1) / a.tn, (a.M + BM - 1) / BM, zsplit);
    k_tc_gemm3<<<grid, THREADS, Cfg3::SMEM, s>>>(ma, mb, mal, mbl, a);
    note_launch();
    return cudaGetLastError();
  }
  if (mode == Mode::Bf16) {  // the converting kernel keeps its full tile width
    TcArgs a = a0;
    a.tn = BN16;
    return launch_kernel(k_tc_gemm16, Cfg16::SMEM, BN16, a, A, lda, B, ldb, zsplit, s);
  }
  if (a0.N > 128) return launch_kernel(k_tc_gemm<256>, Cfg<256>::SMEM, 256, a0, A, lda, B, ldb, zsplit, s);
  return launch_kernel(k_tc_gemm<128>, Cfg<128>::SMEM, 128, a0, A, lda, B, ldb, zsplit, s);
}

}  // namespace tc
}  // namespace kfac
