// Split-precision complex GEMM on the tcgen05 tensor cores (sm_103a).
//
// A complex product C = op(A) op(B) (M x K times K x N) becomes one real GEMM on the embedding
//   A_big = [[Ar, -Ai], [Ai, Ar]]  (2M x 2K),   B_big = [Br; Bi]  (2K x N),   C_big = [Cr; Ci],
// and each FP64 value x is split into two BF16 terms x ~ hi + lo (hi = bf16(x), lo = bf16(x - hi));
// the three leading products hi*hi + hi*lo + lo*hi are obtained by tripling K:
//   A3 = [A_hi | A_hi | A_lo],  B3 = [B_hi ; B_lo ; B_hi]   (K3 = 6K),  C_big = A3 B3,
// accumulated in FP32.  Operands are prepared K-major (A3 rows x K3, B3^T rows x K3) by tiled
// kernels; the GEMM kernel below is a plain BF16 x BF16 -> FP32 tcgen05 GEMM:
//   * one CTA per 128 x BN output tile (BN = 128 or 256), 6 warps: warp 0 issues TMA loads
//     (128B-swizzled 128 x 64 and BN x 64 tiles into a 4-stage ring), warp 1 allocates BN TMEM
//     columns and one of its threads issues tcgen05.mma (M = 128, N = BN, K = 16, BF16 in, FP32
//     accumulator in TMEM), warps 2..5 read the accumulator with tcgen05.ld and store FP32 rows;
//   * full / empty mbarriers per stage (TMA transaction bytes / tcgen05.commit), one more for the
//     finished accumulator; every wait is bounded: on timeout the CTA raises DEV_TIMEOUT in the
//     error word, the other roles stop, outstanding TMA loads are drained (bounded) and the TMEM
//     columns are released before the CTA exits.
//   * TF32 operands (kind::tf32, the TF32x3 split): the tensor cores add each MMA's products into the
//     FP32 accumulator with a truncating alignment, a bias of order 2^-24 |acc| per MMA that grows
//     linearly with K (measured: 1e-7 K relative to |a| |b| sqrt(K) with one accumulator, above the
//     split's own 2^-22).  So each K tile (four MMAs) is accumulated from zero in one of two TMEM
//     buffers, alternately, and the epilogue warps add the finished tile into FP32 registers with
//     round-to-nearest while the next tile is multiplied into the other buffer (accfull / accfree
//     mbarriers per buffer).  The bias is then that of four MMAs per tile; what remains is the
//     FP32 rounding of the tile sum, ~2^-24 sqrt(number of tiles) (measured 6e-7 .. 3e-6 for K = 32
//     .. 1200, against 1.4e-5 at K = 162 with one accumulator).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "prof.cuh"
#include "tc_gemm.cuh"

namespace ipeps {
namespace tc {

constexpr int BM = 128, STAGES = 4, THREADS = 192;
constexpr int ROW_BYTES = 128;                             // one 128-byte swizzled row per K tile
constexpr uint32_t A_BYTES = BM * ROW_BYTES;               // 16 KB A tile per stage
// Operand type of the real GEMM: OP_BF16 (tcgen05 kind::f16 with BF16 operands) or OP_TF32
// (kind::tf32).  A K tile is one 128-byte row per operand row: 64 BF16 or 32 TF32 values; one MMA
// covers 32 bytes of K (16 BF16 or 8 TF32), four per tile.
constexpr int OP_BF16 = 0, OP_TF32 = 1;
template <int OPT> struct OpCfg {
  static constexpr int ELEM = OPT == OP_TF32 ? 4 : 2;
  static constexpr int BK = ROW_BYTES / ELEM;              // K elements per tile
  static constexpr uint32_t FMT = OPT == OP_TF32 ? 2u : 1u;   // instruction-descriptor A/B format
};
// per output-tile width BN (128 or 256): B tile bytes, shared memory, TMEM columns
template <int BN, int OPT> struct TileCfg {
  static constexpr uint32_t B_BYTES = BN * ROW_BYTES;
  static constexpr uint32_t SMEM_BYTES = STAGES * (A_BYTES + B_BYTES) + 1024 + 256;
  // TF32: two accumulator buffers of BN columns (per-tile accumulation, BN = 128 only)
  static_assert(OPT != OP_TF32 || BN == 128, "TF32 tiles are 128 wide");
  static constexpr bool CHUNKED = OPT == OP_TF32;
  static constexpr uint32_t TMEM_COLS = CHUNKED ? 2 * BN : BN;
  // instruction descriptor: A and B of the operand type (same for both, K-major), FP32
  // accumulator, M = 128, N = BN
  static constexpr uint32_t IDESC = (1u << 4)                  // D format F32
                                    | (OpCfg<OPT>::FMT << 7)   // A format
                                    | (OpCfg<OPT>::FMT << 10)  // B format
                                    | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
};
constexpr long long SPIN_LIMIT = 1LL << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; returns false on timeout or when another role has aborted
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  for (long long it = 0; it < SPIN_LIMIT; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255) == 255 && *abort_flag) return false;
  }
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x,
                                            int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}
// shared-memory matrix descriptor: K-major operand tile written by TMA with 128-byte swizzle,
// rows of 128 bytes, 8-row core-matrix groups 1024 bytes apart (tile base 1024-byte aligned)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                  // leading-dimension byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                  // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return d;
}
template <int BN, int OPT>
__global__ void __launch_bounds__(THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               float* __restrict__ C, long long ldc, long long strideC, int ktiles, unsigned* err,
               const int* skip, int skip_mod) {
  // skipped problems: the whole CTA leaves before any barrier, TMA load or TMEM allocation
  if (skipped(skip, skip_mod, (int)blockIdx.z)) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const uint32_t sA = smem_u32(smem);
  using Cfg = TileCfg<BN, OPT>;
  constexpr int BK = OpCfg<OPT>::BK;
  const uint32_t sB = sA + STAGES * A_BYTES;
  unsigned char* tail = smem + STAGES * (A_BYTES + Cfg::B_BYTES);
  // full[STAGES], empty[STAGES], done, accfull[2], accfree[2]
  uint64_t* bars = reinterpret_cast<uint64_t*>(tail);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tail + 8 * (2 * STAGES + 5));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * STAGES, done_bar = full0 + 16 * STAGES;
  const uint32_t accfull0 = done_bar + 8, accfree0 = done_bar + 24;
  constexpr bool CHUNKED = Cfg::CHUNKED;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM, bz = blockIdx.z;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done_bar, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(accfull0 + 8 * b, 1);
      mbar_init(accfree0 + 8 * b, 4);       // one arrival per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(Cfg::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int issued = 0;
    for (int kt = 0; kt < ktiles; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, abort_flag)) {
        *abort_flag = 1;
        atomicOr(err, (unsigned)DEV_TIMEOUT);
        break;
      }
      mbar_expect_tx(full0 + 8 * s, A_BYTES + Cfg::B_BYTES);
      tma_load_3d(sA + s * A_BYTES, &tmA, full0 + 8 * s, kt * BK, m0, bz);
      tma_load_3d(sB + s * Cfg::B_BYTES, &tmB, full0 + 8 * s, kt * BK, n0, bz);
      ++issued;
    }
    // drain: every issued load has completed before the CTA may exit (bounded)
    for (int kt = issued > STAGES ? issued - STAGES : 0; kt < issued; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      for (long long it = 0; it < SPIN_LIMIT && !mbar_try(full0 + 8 * s, ph); ++it) {
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    bool ok = true;
    for (int kt = 0; kt < ktiles; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      const int buf = CHUNKED ? (kt & 1) : 0;
      // per-tile accumulation: the buffer's previous tile (kt - 2) has been read by the epilogue
      if (CHUNKED && kt >= 2 && !mbar_wait(accfree0 + 8 * buf, (uint32_t)((kt - 2) >> 1) & 1u, abort_flag)) {
        *abort_flag = 1;
        atomicOr(err, (unsigned)DEV_TIMEOUT);
        ok = false;
        break;
      }
      if (!mbar_wait(full0 + 8 * s, ph, abort_flag)) {
        *abort_flag = 1;
        atomicOr(err, (unsigned)DEV_TIMEOUT);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t da = smem_desc(sA + s * A_BYTES), db = smem_desc(sB + s * Cfg::B_BYTES);
#pragma unroll
      for (int k = 0; k < ROW_BYTES / 32; ++k) {
        const uint32_t acc = (k > 0 || (!CHUNKED && kt > 0)) ? 1u : 0u;
        const uint64_t adv = (uint64_t)((k * 32) >> 4);   // 32 bytes along K per MMA
        if constexpr (OPT == OP_TF32) {
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (uint32_t)(buf * BN)),
              "l"(da + adv), "l"(db + adv), "r"(Cfg::IDESC), "r"(acc)
              : "memory");
        } else {
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(da + adv), "l"(db + adv), "r"(Cfg::IDESC), "r"(acc)
              : "memory");
        }
      }
      // the stage is free once these MMAs have read it
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       empty0 + 8 * s)
                   : "memory");
      if (CHUNKED)   // this tile's accumulation is complete
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         accfull0 + 8 * buf)
                     : "memory");
    }
    (void)ok;
    // accumulator complete (also signalled after an abort, so the epilogue never waits forever)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     done_bar)
                 : "memory");
  } else if (warp >= 2 && CHUNKED) {
    // ---------------- epilogue, per-tile accumulation: TMEM lanes 32 q .. 32 q + 31 (q = warp % 4);
    // each thread owns one output row and adds every finished tile into BN registers
    const int q = warp & 3;
    float sum[BN];
#pragma unroll
    for (int j = 0; j < BN; ++j) sum[j] = 0.0f;
    bool ok = true;
    for (int kt = 0; kt < ktiles; ++kt) {
      const int buf = kt & 1;
      bool got = mbar_wait(accfull0 + 8 * buf, (uint32_t)(kt >> 1) & 1u, abort_flag);
      got = __all_sync(0xffffffffu, got && !*abort_flag);
      if (!got) {
        if (lane == 0) {
          *abort_flag = 1;
          atomicOr(err, (unsigned)DEV_TIMEOUT);
        }
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * BN + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
            "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
            "%28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
              "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
              "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
              "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 32; ++j) sum[c0 + j] = __fadd_rn(sum[c0 + j], __uint_as_float(r[j]));
      }
      // the buffer may be overwritten by tile kt + 2
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(accfree0 + 8 * buf);
    }
    if (ok) {
      float* crow = C + (long long)bz * strideC + (long long)(m0 + 32 * q + lane) * ldc + n0;
      float4* dst = reinterpret_cast<float4*>(crow);
#pragma unroll
      for (int j = 0; j < BN / 4; ++j)
        dst[j] = make_float4(sum[4 * j], sum[4 * j + 1], sum[4 * j + 2], sum[4 * j + 3]);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: TMEM lanes (32 q .. 32 q + 31) of warp quarter q = warp % 4
    const int q = warp & 3;
    bool ok = mbar_wait(done_bar, 0, abort_flag);
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicOr(err, (unsigned)DEV_TIMEOUT);
    }
    // warp-uniform decision: tcgen05.ld is .sync.aligned
    ok = __all_sync(0xffffffffu, ok && !*abort_flag);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const int row = m0 + 32 * q + lane;
      float* crow = C + (long long)bz * strideC + (long long)row * ldc + n0;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
            "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
            "%28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
              "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
              "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
              "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float4* dst = reinterpret_cast<float4*>(crow + c0);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          dst[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                               __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    // after an abort the issued MMAs may still be running: wait (bounded) for their commit before
    // the columns are released; on the normal path this phase has already completed
    if (lane == 0)
      for (long long it = 0; it < SPIN_LIMIT && !mbar_try(done_bar, 0); ++it) {
      }
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS)
                 : "memory");
  }
}

// ----------------------------------------------------------------------------- operand preparation
// x ~ hi + lo with hi, lo in the operand type: BF16 (8 significant bits each) or TF32 (11 each).
__device__ __forceinline__ void split_term(double x, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
  *hi = h;
  *lo = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
}
// TF32 value of an FP32 number: round to nearest (ties to even) at mantissa bit 13 and clear the
// 13 low bits; the tensor cores read the 19 high bits of the 32-bit word
__device__ __forceinline__ float to_tf32(float f) {
  unsigned u = __float_as_uint(f);
  u += 0x0FFFu + ((u >> 13) & 1u);
  return __uint_as_float(u & 0xFFFFE000u);
}
__device__ __forceinline__ void split_term(double x, float* hi, float* lo) {
  const float h = to_tf32((float)x);
  *hi = h;
  *lo = to_tf32((float)(x - (double)h));
}

// The operands are prepared tile by tile: a 32 x 32 tile of op(A) (rows x K) or of op(B)^T
// (columns x K) is read with coalesced loads along whichever index is contiguous in memory, held
// in shared memory, and written out along K, where each complex element becomes its 12 (A) or 6 (B)
// entries of the operand type T.  Grid: (K tiles, row tiles, batch), so no integer division per
// element.  Columns c >= 6K of both operands are zeroed by the host; rows beyond 2M (A3) or N (B3)
// only feed output entries that are never read.
constexpr int PT = 32;

// tile[r][k] = element (row0 + r, k0 + k) of the operand seen as rows x K, stored either
// K-contiguous (P[row * ld + k]) or row-contiguous (P[k * ld + row]); conjugated for OP_C
__device__ __forceinline__ void load_tile(cplx (*tile)[PT + 1], const cplx* P, long long ld, bool kcontig,
                                          bool cj, int row0, int k0, int rows, int K) {
  const int tx = threadIdx.x;
  for (int a = threadIdx.y; a < PT; a += blockDim.y) {
    if (kcontig) {
      const int r = row0 + a, k = k0 + tx;
      const cplx v = (r < rows && k < K) ? P[(long long)r * ld + k] : cmk(0.0, 0.0);
      tile[a][tx] = cj ? cconj(v) : v;
    } else {
      const int k = k0 + a, r = row0 + tx;
      const cplx v = (r < rows && k < K) ? P[(long long)k * ld + r] : cmk(0.0, 0.0);
      tile[tx][a] = cj ? cconj(v) : v;
    }
  }
}

// A3[b] (Mp x Kp): row r < M holds [Ar | -Ai], row M + r holds [Ai | Ar]; each 2K-wide segment
// appears as hi, hi, lo.
template <typename T>
__global__ void __launch_bounds__(256) prep_a_kernel(GemmDesc g, T* A3, int Mp, int Kp) {
  __shared__ cplx tile[PT][PT + 1];
  const int b = blockIdx.z, M = g.M, K = g.K;
  if (skipped(g.skip, g.skip_mod, b)) return;
  const int row0 = blockIdx.y * PT, k0 = blockIdx.x * PT;
  const cplx* A = g.Aptr ? g.Aptr[b] : g.A + (long long)b * g.sA;
  // op(A)[r][k]: OP_N reads A[r * lda + k]; OP_T and OP_C read A[k * lda + r]
  load_tile(tile, A, g.lda, g.opA == OP_N, g.opA == OP_C, row0, k0, M, K);
  __syncthreads();
  const int k = k0 + threadIdx.x;
  if (k >= K) return;
  for (int a = threadIdx.y; a < PT; a += blockDim.y) {
    const int r = row0 + a;
    if (r >= M) break;
    const cplx v = tile[a][threadIdx.x];
    T rh, rl, ih, il, mh, ml;
    split_term(v.x, &rh, &rl);
    split_term(v.y, &ih, &il);
    split_term(-v.y, &mh, &ml);
    T* up = A3 + ((long long)b * Mp + r) * Kp;        // row r
    T* dn = A3 + ((long long)b * Mp + M + r) * Kp;    // row M + r
    up[k] = rh;          up[K + k] = mh;
    up[2 * K + k] = rh;  up[3 * K + k] = mh;
    up[4 * K + k] = rl;  up[5 * K + k] = ml;
    dn[k] = ih;          dn[K + k] = rh;
    dn[2 * K + k] = ih;  dn[3 * K + k] = rh;
    dn[4 * K + k] = il;  dn[5 * K + k] = rl;
  }
}

// B3t[b] (Np x Kp), row j = column j of B3 = [B_hi; B_lo; B_hi] with B_big = [Br; Bi] (2K x N)
template <typename T>
__global__ void __launch_bounds__(256) prep_b_kernel(GemmDesc g, T* B3t, int Np, int Kp) {
  __shared__ cplx tile[PT][PT + 1];
  const int b = blockIdx.z, N = g.N, K = g.K;
  if (skipped(g.skip, g.skip_mod, b)) return;
  const int row0 = blockIdx.y * PT, k0 = blockIdx.x * PT;
  const cplx* B = g.Bptr ? g.Bptr[b] : g.B + (long long)b * g.sB;
  // op(B)^T[j][k] = op(B)[k][j]: OP_N reads B[k * ldb + j]; OP_T and OP_C read B[j * ldb + k]
  load_tile(tile, B, g.ldb, g.opB != OP_N, g.opB == OP_C, row0, k0, N, K);
  __syncthreads();
  const int k = k0 + threadIdx.x;
  if (k >= K) return;
  for (int a = threadIdx.y; a < PT; a += blockDim.y) {
    const int j = row0 + a;
    if (j >= N) break;
    const cplx v = tile[a][threadIdx.x];
    T rh, rl, ih, il;
    split_term(v.x, &rh, &rl);
    split_term(v.y, &ih, &il);
    T* row = B3t + ((long long)b * Np + j) * Kp;
    row[k] = rh;          row[K + k] = ih;
    row[2 * K + k] = rl;  row[3 * K + k] = il;
    row[4 * K + k] = rh;  row[5 * K + k] = ih;
  }
}

// C[b][i][j] = alpha (C32[i][j] + i C32[M + i][j]) + beta C[b][i][j]; grid (column chunks, rows, batch)
__global__ void __launch_bounds__(256) gather_c_kernel(GemmDesc g, const float* C32, int Mp, int Np) {
  const int b = blockIdx.z, i = blockIdx.y;
  if (skipped(g.skip, g.skip_mod, b)) return;
  const float* top = C32 + ((long long)b * Mp + i) * Np;
  const float* bot = C32 + ((long long)b * Mp + g.M + i) * Np;
  cplx* Cb = g.Cptr ? g.Cptr[b] : g.C + (long long)b * g.sC;
  cplx* crow = Cb + (long long)i * g.ldc;
  const bool use_beta = g.beta.x != 0.0 || g.beta.y != 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < g.N; j += gridDim.x * blockDim.x) {
    cplx r = cmul(g.alpha, cmk((double)top[j], (double)bot[j]));
    if (use_beta) r = cadd(r, cmul(g.beta, crow[j]));
    crow[j] = r;
  }
}

// ----------------------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_encode_mu;

static int encoder(PFN_cuTensorMapEncodeTiled_v12000* out) {
  std::lock_guard<std::mutex> lk(g_encode_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return cuda_fail(e != cudaSuccess ? e : cudaErrorNotSupported, "cuTensorMapEncodeTiled lookup",
                       __FILE__, __LINE__);
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  *out = g_encode;
  return 0;
}

// 3-D map over [batch][rows][Kp] of the operand type with a (128-byte x box_rows x 1) box,
// 128-byte swizzle
template <int OPT>
static int make_map(CUtensorMap* map, const void* base, int rows, int Kp, int batch, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc;
  if (int rc = encoder(&enc)) return rc;
  constexpr int E = OpCfg<OPT>::ELEM;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * E, (cuuint64_t)rows * Kp * E};
  cuuint32_t box[3] = {(cuuint32_t)OpCfg<OPT>::BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, OPT == OP_TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cuda_fail(cudaErrorInvalidValue, "cuTensorMapEncodeTiled", __FILE__, __LINE__);
  return 0;
}

static inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// output-tile width: 256 (twice the reuse of each A tile) for wide products whose own tiles alone
// fill the SMs.  The choice depends on the problem's shape only, never on the batch size, so that
// an instance gets the same arithmetic (the same MMA shapes) alone and in any batch.
static int pick_bn(int M, int N) {
  const long long tiles256 = (long long)(round_up(2 * M, BM) / BM) * (round_up(N, 256) / 256);
  return (N > 128 && tiles256 >= 152) ? 256 : 128;
}

// ---- tile-width autotuner.  The output-tile width does not enter the arithmetic (every output is
// the same K-ordered sum of the same MMA products whatever N the instruction has), so it is picked by
// timing: the first product of each (M, N, K) shape runs with BN = 128 and 256, three timed
// launches each after one warm-up, and the faster width serves every later product of that shape,
// in any batch.  IPEPS_TUNE=0 uses the pick_bn heuristic instead, IPEPS_TUNE=128 or 256 forces that
// width (tests compare the two); tuning is also skipped while the stream is being captured (the
// heuristic serves until the shape is tuned) and for products too narrow for a 256 tile.
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int>, int> g_tuned_bn;

static int tune_mode() {     // 1: tune; 0: heuristic; 128 / 256: forced width
  static const int mode = [] {
    const char* e = std::getenv("IPEPS_TUNE");
    if (!e || !e[0]) return 1;
    const int v = std::atoi(e);
    return (v == 0 || v == 128 || v == 256) ? v : 1;
  }();
  return mode;
}

int tuned_tile_width(int M, int N, int K) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned_bn.find(std::make_tuple(M, N, K));
  return it == g_tuned_bn.end() ? 0 : it->second;
}

template <int OPT>
static int gemm_raw(const void* A3, const void* B3t, float* C32, int Mp, int Np, int ncols, int Kp, int batch,
                    int bn, double algo_flops, unsigned* err, cudaStream_t st, const int* skip, int skip_mod);

// returns the tile width for this BF16 product, tuning it on the prepared operands if needed
static int tile_width(int M, int N, int K, const void* A3, const void* B3, float* C32, int Mp, int Np, int Kp,
                      int batch, unsigned* err, cudaStream_t st, const int* skip, int skip_mod) {
  const int heuristic = pick_bn(M, N), mode = tune_mode();
  if (N <= 128) return 128;
  if (mode == 128 || mode == 256) return mode;
  if (mode == 0) return heuristic;
  const auto key = std::make_tuple(M, N, K);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned_bn.find(key);
    if (it != g_tuned_bn.end()) return it->second;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return heuristic;
  }
  cudaEvent_t e0, e1;
  IPEPS_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError(), "tune events", __FILE__, __LINE__);
  }
  float best_ms = 0.0f;
  int best = heuristic, rc = 0;
  for (int bn : {128, 256}) {
    float ms = 0.0f;
    rc = gemm_raw<OP_BF16>(A3, B3, C32, Mp, Np, N, Kp, batch, bn, -1.0, err, st, skip, skip_mod);
    if (!rc && cudaEventRecord(e0, st) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "tune", __FILE__, __LINE__);
    for (int r = 0; r < 3 && !rc; ++r)
      rc = gemm_raw<OP_BF16>(A3, B3, C32, Mp, Np, N, Kp, batch, bn, -1.0, err, st, skip, skip_mod);
    if (!rc && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = cuda_fail(cudaGetLastError(), "tune timing", __FILE__, __LINE__);
    if (rc) break;
    if (bn == 128 || ms < best_ms) { best_ms = ms; best = bn; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return -rc;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned_bn[key] = best;
  return best;
}

static int k_tile(int op) { return op == SPLIT_TF32 ? OpCfg<OP_TF32>::BK : OpCfg<OP_BF16>::BK; }
static int elem_bytes(int op) { return op == SPLIT_TF32 ? 4 : 2; }

size_t split_workspace_bytes(int M, int N, int K, int batch, int op) {
  const size_t Mp = round_up(2 * M, BM), Np = round_up(N, 256), Kp = round_up(6 * K, k_tile(op));
  return (Mp * Kp + Np * Kp) * elem_bytes(op) * batch + Mp * Np * 4 * batch + 3 * 1024;
}

template <int BN, int OPT>
static int launch_tc(const CUtensorMap& mA, const CUtensorMap& mB, float* C32, int Mp, int Np, int ncols,
                     int Kp, int batch, double algo_flops, unsigned* err, const int* skip, int skip_mod,
                     cudaStream_t st) {
  using Cfg = TileCfg<BN, OPT>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(tc_gemm_kernel<BN, OPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Cfg::SMEM_BYTES);
  });
  IPEPS_CUDA_TRY(attr_err);
  // output tiles over the first ncols columns (C32 rows are Np >= round_up(ncols, BN) wide)
  dim3 grid((ncols + BN - 1) / BN, Mp / BM, batch);
  const double flops = 2.0 * Mp * (double)grid.x * BN * Kp * batch;     // executed on the tensor pipe
  prof_add_tc_executed(flops);
  IPEPS_LAUNCH(K_TC_GEMM, algo_flops > 0.0 ? algo_flops : flops, st,
               (tc_gemm_kernel<BN, OPT><<<grid, THREADS, Cfg::SMEM_BYTES, st>>>(
                   mA, mB, C32, Np, (long long)Mp * Np, Kp / OpCfg<OPT>::BK, err, skip, skip_mod)));
  IPEPS_CUDA_TRY(cudaGetLastError());
  return 0;
}

template <int OPT>
static int gemm_raw(const void* A3, const void* B3t, float* C32, int Mp, int Np, int ncols, int Kp, int batch,
                    int bn, double algo_flops, unsigned* err, cudaStream_t st, const int* skip, int skip_mod) {
  if ((bn != 128 && bn != 256) || Mp % BM || Np % 128 || ncols < 1 || round_up(ncols, bn) > Np ||
      Kp % OpCfg<OPT>::BK || batch < 1 || batch > 65535)
    return cuda_fail(cudaErrorInvalidValue, "tc gemm shape", __FILE__, __LINE__);
  if (((uintptr_t)A3 & 15) || ((uintptr_t)B3t & 15) || ((uintptr_t)C32 & 15))
    return cuda_fail(cudaErrorInvalidValue, "tc gemm alignment", __FILE__, __LINE__);
  CUtensorMap mA, mB;
  if (int rc = make_map<OPT>(&mA, A3, Mp, Kp, batch, BM)) return rc;
  if (int rc = make_map<OPT>(&mB, B3t, Np, Kp, batch, bn)) return rc;
  if constexpr (OPT == OP_TF32) {
    if (bn != 128) return cuda_fail(cudaErrorInvalidValue, "tc gemm tf32 tile width", __FILE__, __LINE__);
    return launch_tc<128, OPT>(mA, mB, C32, Mp, Np, ncols, Kp, batch, algo_flops, err, skip, skip_mod, st);
  } else {
    return bn == 256
               ? launch_tc<256, OPT>(mA, mB, C32, Mp, Np, ncols, Kp, batch, algo_flops, err, skip, skip_mod, st)
               : launch_tc<128, OPT>(mA, mB, C32, Mp, Np, ncols, Kp, batch, algo_flops, err, skip, skip_mod, st);
  }
}

int gemm_bf16_raw(const void* A3, const void* B3t, float* C32, int Mp, int Np, int Kp, int batch,
                  int bn, double algo_flops, unsigned* err, cudaStream_t st, const int* skip,
                  int skip_mod) {
  return gemm_raw<OP_BF16>(A3, B3t, C32, Mp, Np, Np, Kp, batch, bn, algo_flops, err, st, skip, skip_mod);
}

template <typename T, int OPT>
static int zgemm_split_t(const GemmDesc& g, void* work, size_t work_bytes, unsigned* err, cudaStream_t st) {
  const int op = OPT == OP_TF32 ? SPLIT_TF32 : SPLIT_BF16;
  // operand / product layout: rows of B3 and C32 padded to 256 when a 256-wide tile may be used
  const int Mp = round_up(2 * g.M, BM), Kp = round_up(6 * g.K, OpCfg<OPT>::BK);
  const int Np = (OPT == OP_BF16 && g.N > 128) ? round_up(g.N, 256) : round_up(g.N, 128);
  if (split_workspace_bytes(g.M, g.N, g.K, g.batch, op) > work_bytes)
    return cuda_fail(cudaErrorInvalidValue, "split workspace too small", __FILE__, __LINE__);
  char* w = (char*)(((uintptr_t)work + 1023) & ~(uintptr_t)1023);
  T* A3 = (T*)w;
  w += ((size_t)Mp * Kp * sizeof(T) * g.batch + 1023) & ~(size_t)1023;
  T* B3 = (T*)w;
  w += ((size_t)Np * Kp * sizeof(T) * g.batch + 1023) & ~(size_t)1023;
  float* C32 = (float*)w;
  if (g.batch > 65535 || g.M > 65535) return cuda_fail(cudaErrorInvalidValue, "split gemm grid", __FILE__, __LINE__);
  // zero K padding (columns 6K .. Kp) of both operands; the GEMM reads it
  if (Kp > 6 * g.K) {
    const size_t pitch = (size_t)Kp * sizeof(T), width = (size_t)(Kp - 6 * g.K) * sizeof(T);
    IPEPS_CUDA_TRY(cudaMemset2DAsync(A3 + 6 * g.K, pitch, 0, width, (size_t)Mp * g.batch, st));
    IPEPS_CUDA_TRY(cudaMemset2DAsync(B3 + 6 * g.K, pitch, 0, width, (size_t)Np * g.batch, st));
  }
  const dim3 pblk(PT, 8);
  const dim3 pa((g.K + PT - 1) / PT, (g.M + PT - 1) / PT, g.batch);
  const dim3 pb((g.K + PT - 1) / PT, (g.N + PT - 1) / PT, g.batch);
  IPEPS_LAUNCH(K_TC_PREP, 0, st, prep_a_kernel<T><<<pa, pblk, 0, st>>>(g, A3, Mp, Kp));
  IPEPS_LAUNCH(K_TC_PREP, 0, st, prep_b_kernel<T><<<pb, pblk, 0, st>>>(g, B3, Np, Kp));
  IPEPS_CUDA_TRY(cudaGetLastError());
  const double algo = 8.0 * g.M * (double)g.N * g.K * g.batch;   // the complex product's own flops
  int bn = 128;
  if constexpr (OPT == OP_BF16) {
    bn = tile_width(g.M, g.N, g.K, A3, B3, C32, Mp, Np, Kp, g.batch, err, st, g.skip, g.skip_mod);
    if (bn < 0) return -bn;
  }
  if (int rc = gemm_raw<OPT>(A3, B3, C32, Mp, Np, g.N, Kp, g.batch, bn, algo, err, st, g.skip, g.skip_mod)) return rc;
  const dim3 gc((g.N + 255) / 256, g.M, g.batch);
  IPEPS_LAUNCH(K_TC_PREP, 0, st, gather_c_kernel<<<gc, 256, 0, st>>>(g, C32, Mp, Np));
  IPEPS_CUDA_TRY(cudaGetLastError());
  return 0;
}

int zgemm_split(const GemmDesc& g, int op, void* work, size_t work_bytes, unsigned* err, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.batch <= 0) return 0;
  if (op == SPLIT_TF32) return zgemm_split_t<float, OP_TF32>(g, work, work_bytes, err, st);
  return zgemm_split_t<__nv_bfloat16, OP_BF16>(g, work, work_bytes, err, st);
}

}  // namespace tc
}  // namespace ipeps
