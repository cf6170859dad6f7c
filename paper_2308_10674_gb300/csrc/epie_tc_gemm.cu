// epie_tc_gemm.cu -- hand-written tcgen05 GEMM for the DFT-as-GEMM path.
//
//   D[M x Nn] (fp32, row pitch ldd) = sum over terms t of A_t[M x K] * B_t[Nn x K]^T
//
// A_t and B_t are bf16 (kind::f16) or fp32 read as tf32 (kind::tf32),
// row-major with K contiguous (both operands K-major).  One term is the plain
// product (A0 B0); three terms are the split product A0 B0 + A0 B1 + A1 B0
// (x = x_hi + x_lo), all accumulated in one fp32 accumulator in tensor
// memory.  In the DFT path A is a block of rows of
// interleaved complex values and B the transposed 2N x 2N twiddle matrix, so
// one call is the DFT of every row (Sec. "ePIE Implementation": the
// projection runs through a DFT of 2^n frames).
//
// Kernel design (persistent, one CTA of 192 threads per SM; 128 x BN tiles
// of D, BN = 256, or 128 when Nn is not a multiple of 256):
//   * operand tiles of 128 (A) and BN (B) rows of 128 bytes (64 bf16 or 32
//     fp32 values of K) are fetched by TMA (cp.async.bulk.tensor.2d,
//     128-byte swizzle) into a 4-stage ring in shared memory; mbarrier
//     "full[s]" completes on the copied bytes;
//   * thread 0 of warp 0 issues the copies; thread 0 of warp 1 issues
//     tcgen05.mma (M = 128, N = BN, 32 bytes of the rows per instruction:
//     kind::f16 with bf16 or kind::tf32; fp32 accumulation) from
//     shared-memory descriptors, and tcgen05.commit on "empty[s]" returns
//     the stage to the producer;
//   * two BN-column accumulators alternate in tensor memory; after a tile's
//     last k-block a commit completes "acc_full[b]", warps 2-5 read the rows
//     of their TMEM lane quadrant with tcgen05.ld.32x32b, stage them through
//     shared memory and store whole 128-byte row segments (or, for the DFT
//     path's row passes, store the product of whole frames transposed and
//     split into bf16 hi / lo straight from the registers), then arrive on
//     "acc_empty[b]", while the MMAs of the next tile run.
// Every wait is bounded by %globaltimer (2 s).  On expiry the kernel sets
// FLAG_TC_TIMEOUT in the status word, stops, lets its issued copies land and
// its MMAs finish (bounded again), frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>

#include "../../include/epie.h"
#include "epie_fft.cuh"
#include "epie_internal.h"

namespace epie {

namespace {

constexpr int TC_BM = 128, TC_STAGES = 4;
// every operand row of a stage is 128 bytes (one swizzle width): 64 bf16 or
// 32 fp32/tf32 values of K
template <bool TF32>
struct TcElem {
  static constexpr int BYTES = TF32 ? 4 : 2;
  static constexpr int BK = 128 / BYTES;
};
constexpr uint64_t TC_WAIT_NS = 2000000000ull;
// failure injection for the tests of the bounded waits (tc_gemm_inject)
std::atomic<int> g_tc_inject{0};
std::atomic<long long> g_tc_inject_wait_ns{0};

// ---------------------------------------------------------------- PTX wrappers

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}


// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle.  Rows
// are 128 bytes (64 bf16), eight rows form a 1024-byte swizzle atom and the
// atoms follow each other along M/N (stride byte offset 1024).  The leading
// byte offset is unused for a swizzled K-major tile whose K extent is one
// swizzle width.  Bits: start address >> 4 [0,14), LBO >> 4 [16,30),
// SBO >> 4 [32,46), descriptor version 1 [46,48), swizzle mode 2 = 128 B
// [61,64).
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
  return static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4) |
         (static_cast<uint64_t>(1024u >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor: fp32 accumulator [4,6) = 1; A and B format at
// [7,10) and [10,13): bf16 = 1 under kind::f16, tf32 = 2 under kind::tf32;
// both K-major (bits 15, 16 clear); N >> 3 at [17,23), M >> 4 at [24,29).
template <int M, int N, bool TF32>
__host__ __device__ constexpr uint32_t mma_idesc() {
  return (1u << 4) | ((TF32 ? 2u : 1u) << 7) | ((TF32 ? 2u : 1u) << 10) |
         (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

// one MMA over 32 bytes of the operand rows (16 bf16 or 8 tf32 values of K)
template <bool TF32>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                     uint32_t idesc, uint32_t accumulate) {
  if constexpr (TF32)
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 consecutive fp32 columns of this thread's accumulator row
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                   smem_u32(bar))
               : "memory");
}

template <int BN>
struct TcCfg {
  static constexpr uint32_t A_BYTES = TC_BM * 128;
  static constexpr uint32_t B_BYTES = BN * 128;
  static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
  static constexpr size_t OFF_BAR = static_cast<size_t>(TC_STAGES) * STAGE;
  // full[S], empty[S], acc_full[2], acc_empty[2], mma_done; then the TMEM
  // address slot and the abort word
  static constexpr int NBAR = 2 * TC_STAGES + 5;
  // per epilogue warp a 32 x 32 fp32 staging tile, rows padded to 36 floats
  // (16-byte aligned rows; 8 lanes of a quarter-warp touch distinct banks)
  static constexpr int STG_PITCH = 36;
  static constexpr size_t OFF_STG = (OFF_BAR + 8 * NBAR + 16 + 15) / 16 * 16;
  static constexpr size_t STG_BYTES = 32 * STG_PITCH * 4;
  static constexpr size_t SMEM = 1024 + OFF_STG + 4 * STG_BYTES;
  static_assert(OFF_STG % 16 == 0, "staging tiles are read as float4");
  static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "swizzle atoms stay aligned");
};

constexpr int TC_THREADS = 192;  // warp 0 TMA, warp 1 MMA (owns TMEM), warps 2-5 epilogue

// Persistent: CTA b takes tiles b, b + gridDim.x, ... (tile t = row block
// t / n_tiles, column block t % n_tiles, so neighbouring CTAs share the row
// block in L2).  Two accumulators of BN columns alternate in TMEM: the
// epilogue drains tile i while the MMAs of tile i + 1 run.
template <int BN, bool TF32>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                   const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1,
                   float *__restrict__ D, int ldd, int K, int terms, int m_tiles, int n_tiles,
                   int *err_flag, uint64_t wait_ns, int inject, int fn,
                   __nv_bfloat162 *__restrict__ Thi, __nv_bfloat162 *__restrict__ Tlo) {
  using C = TcCfg<BN>;
  extern __shared__ uint8_t smem_raw[];
  // 128-byte-swizzled tiles want 1024-byte alignment
  uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);
  uint64_t *empty = full + TC_STAGES;
  uint64_t *acc_full = empty + TC_STAGES;
  uint64_t *acc_empty = acc_full + 2;
  uint64_t *mma_done = acc_empty + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
  volatile int *abort_word = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int BK = TcElem<TF32>::BK;
  const int kb_term = K / BK, nkb = kb_term * terms;
  const int tiles = m_tiles * n_tiles;
  auto fail = [&]() {
    *abort_word = 1;
    atomicOr(err_flag, FLAG_TC_TIMEOUT);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);  // one arrival per epilogue warp
    }
    mbar_init(mma_done, 1);
    *abort_word = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, 2 * BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer: TMA copies of the operand tiles, k-block after k-block
      int it = 0;
      for (int tile = blockIdx.x; tile < tiles && !*abort_word; tile += gridDim.x) {
        const int m0 = (tile / n_tiles) * TC_BM, n0 = (tile % n_tiles) * BN;
        for (int kb = 0; kb < nkb; ++kb) {
          const int s = it % TC_STAGES, u = it / TC_STAGES;
          if (it >= TC_STAGES && !mbar_wait_bounded(&empty[s], (u - 1) & 1, wait_ns)) {
            fail();
            break;
          }
          if (*abort_word) break;
          if (inject && blockIdx.x == 0 && it == 0) {
            // failure injection (tests of the timeout path): the first stage's
            // copies are never issued, so nothing is in flight for it and every
            // wait on it expires after wait_ns
            ++it;
            continue;
          }
          const int t = kb / kb_term, kx = (kb % kb_term) * BK;
          const CUtensorMap *ma = t == 2 ? &mA1 : &mA0;  // terms: A0 B0, A0 B1, A1 B0
          const CUtensorMap *mb = t == 1 ? &mB1 : &mB0;
          uint8_t *sa = smem + static_cast<size_t>(s) * C::STAGE;
          mbar_arrive_expect_tx(&full[s], C::STAGE);
          tma_load_2d(sa, ma, kx, m0, &full[s]);
          tma_load_2d(sa + C::A_BYTES, mb, kx, n0, &full[s]);
          ++it;
        }
      }
      // every issued copy has landed before the CTA can exit
      for (int j = it - TC_STAGES < 0 ? 0 : it - TC_STAGES; j < it; ++j)
        if (!mbar_wait_bounded(&full[j % TC_STAGES], (j / TC_STAGES) & 1, wait_ns)) fail();
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      constexpr uint32_t idesc = mma_idesc<TC_BM, BN, TF32>();
      int it = 0, tl = 0;
      for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++tl) {
        if (*abort_word) break;
        const int b = tl & 1, ub = tl >> 1;
        if (tl >= 2 && !mbar_wait_bounded(&acc_empty[b], (ub - 1) & 1, wait_ns)) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + static_cast<uint32_t>(b * BN);
        bool bad = false;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % TC_STAGES, u = it / TC_STAGES;
          if (!mbar_wait_bounded(&full[s], u & 1, wait_ns)) {
            fail();
            bad = true;
            break;
          }
          tc_fence_after();
          const uint32_t a_addr = smem_u32(smem + static_cast<size_t>(s) * C::STAGE);
          const uint32_t b_addr = a_addr + C::A_BYTES;
#pragma unroll
          for (int k = 0; k < 4; ++k)  // 32 bytes of the 128-byte rows per instruction
            umma<TF32>(acc, sw128_kmajor_desc(a_addr + 32 * k), sw128_kmajor_desc(b_addr + 32 * k),
                       idesc, (kb | k) != 0);
          umma_commit(&empty[s]);
        }
        if (bad) break;
        umma_commit(&acc_full[b]);
      }
      // every issued MMA has finished before the teardown frees the TMEM
      umma_commit(mma_done);
      if (!mbar_wait_bounded(mma_done, 0, wait_ns)) fail();
    }
  } else {
    // ---- epilogue: TMEM -> registers -> global; warp w reads TMEM lanes
    // 32 (w % 4) .. 32 (w % 4) + 31, i.e. rows of that quadrant of the tile
    const int q = warp & 3;
    int tl = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++tl) {
      const int b = tl & 1, ub = tl >> 1;
      bool ok = mbar_wait_bounded(&acc_full[b], ub & 1, wait_ns);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok || *abort_word) {
        if (!ok && lane == 0) fail();
        break;
      }
      tc_fence_after();
      const int m0 = (tile / n_tiles) * TC_BM, n0 = (tile % n_tiles) * BN;
      const uint32_t tq = tmem + static_cast<uint32_t>(b * BN) + (static_cast<uint32_t>(32 * q) << 16);
      if (Thi) {
        // transposed split output: row R = f fn + y of D holds the row y of
        // frame f as interleaved complex values (column 2 x + c); it goes to
        // row f fn + x, column 2 y + c of the next GEMM's operand, as
        // hi = bf16(v) and lo = bf16(v - hi).  Lane l holds row y0 + l, so for
        // each x the warp's stores are 32 consecutive 4-byte (re, im) pairs.
        const long long R = static_cast<long long>(m0) + 32 * q + lane;
        const long long fr = R / fn;
        const int y = static_cast<int>(R - fr * fn);
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
          uint32_t r[32];
          tmem_ld32(tq + c, r);
          const long long row0 = fr * fn + ((n0 + c) >> 1);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float re = __uint_as_float(r[2 * j]), im = __uint_as_float(r[2 * j + 1]);
            const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
            const size_t o = static_cast<size_t>(row0 + j) * fn + y;  // in (re, im) pairs
            Thi[o] = h;
            if (Tlo) Tlo[o] = __floats2bfloat162_rn(re - __low2float(h), im - __high2float(h));
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[b]);
        continue;
      }
      // lane l holds row l of the warp's 32 rows; through the staging tile,
      // lanes 8i..8i+7 then store 128 contiguous bytes of one row
      float *stg = reinterpret_cast<float *>(smem + C::OFF_STG + (warp - 2) * C::STG_BYTES);
      const int sr = lane >> 3, sc = (lane & 7) * 4;
      float *dbase = D + static_cast<size_t>(m0 + 32 * q) * ldd + n0;
#pragma unroll 1
      for (int c = 0; c < BN; c += 32) {
        uint32_t r[32];
        tmem_ld32(tq + c, r);
#pragma unroll
        for (int j = 0; j < 32; j += 4)
          *reinterpret_cast<float4 *>(stg + lane * C::STG_PITCH + j) =
              make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                          __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int row = 4 * i + sr;
          *reinterpret_cast<float4 *>(dbase + static_cast<size_t>(row) * ldd + c + sc) =
              *reinterpret_cast<const float4 *>(stg + row * C::STG_PITCH + sc);
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * BN);
  }
}

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder(std::string *err) {
  static EncodeTiled fn = nullptr;
  if (fn) return fn;
  void *p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    *err = "cuTensorMapEncodeTiled is not available from the driver";
    return nullptr;
  }
  fn = reinterpret_cast<EncodeTiled>(p);
  return fn;
}

// rows x K values (bf16, or fp32 read as tf32), row-major; box = box_rows x
// (128 bytes of K), 128-byte swizzle
bool make_map(CUtensorMap *m, const void *base, long long rows, int K, int box_rows, bool tf32,
              std::string *err) {
  EncodeTiled enc = encoder(err);
  if (!enc) return false;
  const int es = tf32 ? 4 : 2;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(K) * es};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(128 / es), static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void *>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *err = "cuTensorMapEncodeTiled failed (" + std::to_string(static_cast<int>(r)) + ")";
    return false;
  }
  return true;
}

// where the product goes: fp32 D (row pitch ldd), or, when thi is set, the
// rows of frames of side fn transposed and split into bf16 hi / lo pairs
struct TcOut {
  float *D = nullptr;
  int ldd = 0;
  int fn = 0;
  __nv_bfloat162 *thi = nullptr, *tlo = nullptr;
};

template <int BN, bool TF32>
cudaError_t launch_tc(const CUtensorMap &a0, const CUtensorMap &a1, const CUtensorMap &b0,
                      const CUtensorMap &b1, const TcOut &out, long long M, int Nn, int K,
                      int terms, int *err_flag, uint64_t wait_ns, int inject, cudaStream_t st) {
  using C = TcCfg<BN>;
  static int attr_dev = -1, sms = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<BN, TF32>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(C::SMEM));
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  const int m_tiles = static_cast<int>(M / TC_BM), n_tiles = Nn / BN;
  const long long tiles = static_cast<long long>(m_tiles) * n_tiles;
  const int grid = static_cast<int>(tiles < sms ? tiles : sms);  // one CTA per SM
  tc_gemm_kernel<BN, TF32><<<grid, TC_THREADS, C::SMEM, st>>>(
      a0, a1, b0, b1, out.D, out.ldd, K, terms, m_tiles, n_tiles, err_flag, wait_ns, inject,
      out.fn, out.thi, out.tlo);
  return cudaGetLastError();
}

int tc_gemm(const void *A0, const void *A1, const void *B0, const void *B1, const TcOut &out,
            long long M, int Nn, int K, int terms, bool tf32, int *err_flag, cudaStream_t st,
            std::string *err) {
  const int BN = Nn % 256 == 0 ? 256 : 128;
  const int bk = tf32 ? TcElem<true>::BK : TcElem<false>::BK;
  const bool split = out.thi != nullptr;
  if (!A0 || !B0 || (!split && !out.D) || !err_flag || (terms != 1 && terms != 3) ||
      (terms == 3 && (!A1 || !B1))) {
    *err = "null operand, or terms not 1 or 3";
    return EPIE_EINVAL;
  }
  if (M <= 0 || M % TC_BM || Nn <= 0 || Nn % 128 || K <= 0 || K % bk ||
      (!split && (out.ldd < Nn || out.ldd % 4)) || (M / TC_BM) * (Nn / 128) > 0x7fffffffLL) {
    *err = "M must be a positive multiple of 128, Nn of 128, K of " + std::to_string(bk) +
           "; ldd >= Nn and a multiple of 4";
    return EPIE_EINVAL;
  }
  // transposed output: whole frames of side fn (a multiple of 32, so a
  // warp's 32 rows lie in one frame), rows of 2 fn values
  if (split && (tf32 || out.fn < 32 || out.fn % 32 || Nn != 2 * out.fn || M % out.fn)) {
    *err = "transposed output: bf16 operands, frame side a multiple of 32, Nn = 2 fn, M = frames x fn";
    return EPIE_EINVAL;
  }
  const void *dst = split ? static_cast<const void *>(out.thi) : static_cast<const void *>(out.D);
  const void *dst2 = split && out.tlo ? static_cast<const void *>(out.tlo) : dst;
  const void *ptrs[6] = {A0, A1 ? A1 : A0, B0, B1 ? B1 : B0, dst, dst2};
  for (const void *p : ptrs)
    if (reinterpret_cast<uintptr_t>(p) % 16) {
      *err = "operands must be 16-byte aligned";
      return EPIE_EINVAL;
    }
  CUtensorMap a0, a1, b0, b1;
  if (!make_map(&a0, A0, M, K, TC_BM, tf32, err) ||
      !make_map(&a1, A1 ? A1 : A0, M, K, TC_BM, tf32, err) ||
      !make_map(&b0, B0, Nn, K, BN, tf32, err) || !make_map(&b1, B1 ? B1 : B0, Nn, K, BN, tf32, err))
    return EPIE_ECUDA;
  uint64_t w = TC_WAIT_NS;
  int inj = 0;
  for (int c = g_tc_inject.load(); c > 0;)
    if (g_tc_inject.compare_exchange_weak(c, c - 1)) {
      inj = 1;
      w = static_cast<uint64_t>(g_tc_inject_wait_ns.load());
      break;
    }
  cudaError_t e;
  if (tf32)
    e = BN == 256 ? launch_tc<256, true>(a0, a1, b0, b1, out, M, Nn, K, terms, err_flag, w, inj, st)
                  : launch_tc<128, true>(a0, a1, b0, b1, out, M, Nn, K, terms, err_flag, w, inj, st);
  else
    e = BN == 256 ? launch_tc<256, false>(a0, a1, b0, b1, out, M, Nn, K, terms, err_flag, w, inj, st)
                  : launch_tc<128, false>(a0, a1, b0, b1, out, M, Nn, K, terms, err_flag, w, inj, st);
  if (e != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return EPIE_ECUDA;
  }
  return EPIE_OK;
}

}  // namespace

void tc_gemm_inject(int count, long long wait_ns) {
  g_tc_inject_wait_ns.store(wait_ns);
  g_tc_inject.store(count);
}

int tc_gemm_bf16(const void *A0, const void *A1, const void *B0, const void *B1, float *D,
                 long long M, int Nn, int K, int ldd, int terms, int *err_flag, cudaStream_t st,
                 std::string *err) {
  TcOut out;
  out.D = D;
  out.ldd = ldd;
  return tc_gemm(A0, A1, B0, B1, out, M, Nn, K, terms, false, err_flag, st, err);
}

int tc_gemm_bf16_tsplit(const void *A0, const void *A1, const void *B0, const void *B1, void *hi,
                        void *lo, long long M, int fn, int K, int terms, int *err_flag,
                        cudaStream_t st, std::string *err) {
  TcOut out;
  out.fn = fn;
  out.thi = static_cast<__nv_bfloat162 *>(hi);
  out.tlo = static_cast<__nv_bfloat162 *>(lo);
  if (!hi) {
    *err = "null output";
    return EPIE_EINVAL;
  }
  return tc_gemm(A0, A1, B0, B1, out, M, 2 * fn, K, terms, false, err_flag, st, err);
}

int tc_gemm_tf32(const float *A0, const float *A1, const float *B0, const float *B1, float *D,
                 long long M, int Nn, int K, int ldd, int terms, int *err_flag, cudaStream_t st,
                 std::string *err) {
  TcOut out;
  out.D = D;
  out.ldd = ldd;
  return tc_gemm(A0, A1, B0, B1, out, M, Nn, K, terms, true, err_flag, st, err);
}

}  // namespace epie
