// epie_fft.cuh -- device building blocks of the fused ePIE kernel:
// complex arithmetic, radix-4/8/16 register DFTs, Stockham passes over
// batches of 1-D transforms held in shared memory, and the PTX wrappers for
// the mbarrier-tracked bulk (TMA) copy of the intensity tile.
//
// Transform convention (paper: DFT forward / back projection on 2^n frames,
// Sec. "ePIE Implementation"): forward X[k] = sum_n x[n] exp(-2 pi i n k / N),
// inverse without the 1/N factor (the caller folds 1/N^2 into the modulus
// replacement).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace epie {

// ------------------------------------------------------------------ complex

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Packed complex add and subtract for the butterflies: one paired-FP32
// instruction (sm_100 family) in place of two scalar ones.  Each lane rounds
// exactly like the scalar operation, and b * (-1) + a is a - b with one
// rounding, so the results are bit-identical to cadd / csub.
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
// a * (c + i s) as a.x (c, s) + a.y (-s, c): two paired-FP32 instructions
// with a component of a broadcast to both lanes, in place of two multiplies
// and two fused multiply-adds
__device__ __forceinline__ float2 cmul_const(float2 a, float c, float s) {
  return __ffma2_rn(make_float2(a.y, a.y), make_float2(-s, c), __fmul2_rn(make_float2(a.x, a.x), make_float2(c, s)));
}

// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos / sin of 2 pi e / 16, written from the half-angle values
// cos(pi/8) = sqrt(2 + sqrt 2)/2, sin(pi/8) = sqrt(2 - sqrt 2)/2, sqrt(2)/2.
__host__ __device__ constexpr float cos16(int e) {
  constexpr float C1 = 0.92387953251128675613f, S1 = 0.38268343236508977173f,
                  H = 0.70710678118654752440f;
  switch (e & 15) {
    case 0: return 1.f;   case 1: return C1;  case 2: return H;   case 3: return S1;
    case 4: return 0.f;   case 5: return -S1; case 6: return -H;  case 7: return -C1;
    case 8: return -1.f;  case 9: return -C1; case 10: return -H; case 11: return -S1;
    case 12: return 0.f;  case 13: return S1; case 14: return H;  default: return C1;
  }
}
__host__ __device__ constexpr float sin16(int e) { return cos16(e - 4); }

// a * W16^E with W16 = exp(-+ 2 pi i / 16) (forward: minus)
template <int E, bool INV>
__device__ __forceinline__ float2 tw16(float2 a) {
  constexpr int e = E & 15;
  if constexpr (e == 0) {
    return a;
  } else if constexpr (e == 4) {
    return mul_mi<INV>(a);
  } else if constexpr (e == 8) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (e == 12) {
    return mul_mi<!INV>(a);
  } else {
    constexpr float c = cos16(e);
    constexpr float s = INV ? sin16(e) : -sin16(e);
    return cmul_const(a, c, s);
  }
}

// ------------------------------------------------------------------ small DFTs (natural order, in place)

template <bool INV>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
  const float2 t0 = padd(a0, a2), t1 = psub(a0, a2);
  const float2 t2 = padd(a1, a3), d = psub(a1, a3);
  a0 = padd(t0, t2);
  a2 = psub(t0, t2);
  // t1 -+ i d: the swapped components stay scalar
  a1 = INV ? make_float2(t1.x - d.y, t1.y + d.x) : make_float2(t1.x + d.y, t1.y - d.x);
  a3 = INV ? make_float2(t1.x + d.y, t1.y - d.x) : make_float2(t1.x - d.y, t1.y + d.x);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
  dft4<INV>(v[0], v[2], v[4], v[6]);  // even part E[k] at v[2k]
  dft4<INV>(v[1], v[3], v[5], v[7]);  // odd part  O[k] at v[2k+1]
  const float2 o0 = v[1], o1 = tw16<2, INV>(v[3]), o2 = tw16<4, INV>(v[5]), o3 = tw16<6, INV>(v[7]);
  const float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  v[0] = padd(e0, o0); v[4] = psub(e0, o0);
  v[1] = padd(e1, o1); v[5] = psub(e1, o1);
  v[2] = padd(e2, o2); v[6] = psub(e2, o2);
  v[3] = padd(e3, o3); v[7] = psub(e3, o3);
}

// 16 = 4 x 4: n = 4m + t, k = k1 + 4 k2;
// X[k1 + 4k2] = sum_t W4^(t k2) W16^(t k1) sum_m x[4m + t] W4^(m k1)
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
#pragma unroll
  for (int t = 0; t < 4; ++t) dft4<INV>(v[t], v[4 + t], v[8 + t], v[12 + t]);
  v[5] = tw16<1, INV>(v[5]);
  v[6] = tw16<2, INV>(v[6]);
  v[7] = tw16<3, INV>(v[7]);
  v[9] = tw16<2, INV>(v[9]);
  v[10] = tw16<4, INV>(v[10]);
  v[11] = tw16<6, INV>(v[11]);
  v[13] = tw16<3, INV>(v[13]);
  v[14] = tw16<6, INV>(v[14]);
  v[15] = tw16<9, INV>(v[15]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // v[4 k1 + k2] holds X[k1 + 4 k2]: transpose the 4x4 index
  float2 t;
  t = v[1];  v[1] = v[4];   v[4] = t;
  t = v[2];  v[2] = v[8];   v[8] = t;
  t = v[3];  v[3] = v[12];  v[12] = t;
  t = v[6];  v[6] = v[9];   v[9] = t;
  t = v[7];  v[7] = v[13];  v[13] = t;
  t = v[11]; v[11] = v[14]; v[14] = t;
}

// cos / sin of 2 pi e / 32 (quarter-wave symmetry from the values at
// e = 0..8: cos(pi/16), cos(pi/8), cos(3 pi/16), ...)
__host__ __device__ constexpr float cos32(int e) {
  constexpr float Q[9] = {1.f,
                          0.980785280403230449126f,
                          0.923879532511286756128f,
                          0.831469612302545237079f,
                          0.707106781186547524401f,
                          0.555570233019602224743f,
                          0.382683432365089771728f,
                          0.195090322016128267848f,
                          0.f};
  const int m = e & 31;
  return m <= 8 ? Q[m] : m <= 16 ? -Q[16 - m] : m <= 24 ? -Q[m - 16] : Q[32 - m];
}
__host__ __device__ constexpr float sin32(int e) { return cos32(e - 8); }

// a * W32^E with W32 = exp(-+ 2 pi i / 32) (forward: minus)
template <int E, bool INV>
__device__ __forceinline__ float2 tw32(float2 a) {
  constexpr int e = E & 31;
  if constexpr ((e & 1) == 0) {
    return tw16<e / 2, INV>(a);
  } else {
    constexpr float c = cos32(e);
    constexpr float s = INV ? sin32(e) : -sin32(e);
    return cmul_const(a, c, s);
  }
}

template <bool INV, int K>
__device__ __forceinline__ void dft32_combine(const float2 (&e)[16], const float2 (&o)[16],
                                              float2 (&lo)[16], float2 (&hi)[16]) {
  if constexpr (K < 16) {
    const float2 t = tw32<K, INV>(o[K]);
    lo[K] = padd(e[K], t);
    hi[K] = psub(e[K], t);
    dft32_combine<INV, K + 1>(e, o, lo, hi);
  }
}

// 32-point DFT of x[0..31] = (lo[0..15], hi[0..15]) in natural order, in
// place (decimation in time: two 16-point DFTs of the even and the odd
// samples, X[k] = E[k] + W32^k O[k], X[k + 16] = E[k] - W32^k O[k])
template <bool INV>
__device__ __forceinline__ void dft32(float2 (&lo)[16], float2 (&hi)[16]) {
  float2 e[16], o[16];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    e[m] = lo[2 * m];
    o[m] = lo[2 * m + 1];
    e[m + 8] = hi[2 * m];
    o[m + 8] = hi[2 * m + 1];
  }
  dft16<INV>(e);
  dft16<INV>(o);
  dft32_combine<INV, 0>(e, o, lo, hi);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
  if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 16) dft16<INV>(v);
  else static_assert(R == 4 || R == 8 || R == 16, "radix 4, 8 or 16");
}

// ------------------------------------------------------------------ shared-memory layouts

// one padding element after every 16 along a padded axis (bank spreading)
__host__ __device__ constexpr int pidx(int x) { return x + (x >> 4); }

// column-major use of a row-major tile: element n of column b at n*ES + off(b)
template <int ES, bool PADB>
struct ColAddr {
  static __device__ __forceinline__ int at(int b, int n) { return n * ES + (PADB ? pidx(b) : b); }
};
// element n of row b in a row-major tile with padded rows of pitch PB
template <int PB>
struct RowAddr {
  static __device__ __forceinline__ int at(int b, int n) { return b * PB + pidx(n); }
};

// ------------------------------------------------------------------ Stockham passes

// One radix-R Stockham pass (span NS -> NS*R) over BATCH transforms of length
// N held in shared memory s (addressing A).  Each of the NT threads takes
// BATCH*(N/R)/NT butterflies; butterfly j of transform b reads elements
// j + r N/R, twiddles them by W_{NS R}^{r (j mod NS)}, runs the radix-R DFT
// and writes element (j - k) R + k + r NS.  Loads finish (barrier) before
// stores, so the pass works in place.  JFAST selects the thread order
// (j fastest for row tiles, b fastest for column tiles).
template <int N, int R, int NS, bool INV, int NT, int BATCH, bool JFAST, class A>
__device__ __forceinline__ void fft_pass(float2 *__restrict__ s, const float2 *__restrict__ tw) {
  constexpr int NJ = N / R;
  constexpr int PER = BATCH * NJ / NT;
  static_assert(PER >= 1 && PER * NT == BATCH * NJ, "butterflies must split evenly");
  float2 v[PER][R];
  int bb[PER], jj[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int u = threadIdx.x + i * NT;
    const int j = JFAST ? (u % NJ) : (u / BATCH);
    const int b = JFAST ? (u / NJ) : (u % BATCH);
    bb[i] = b;
    jj[i] = j;
#pragma unroll
    for (int r = 0; r < R; ++r) v[i][r] = s[A::at(b, j + r * NJ)];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int k = jj[i] & (NS - 1);
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = tw[(r * k) * (N / (NS * R))];
        if (INV) w.y = -w.y;
        v[i][r] = cmul(v[i][r], w);
      }
    }
    dft<R, INV>(v[i]);
    const int base = (jj[i] - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) s[A::at(bb[i], base + r * NS)] = v[i][r];
  }
  __syncthreads();
}

// The last forward pass (radix R, span N/R), a pointwise map of the
// finished spectrum, and the first inverse pass (radix R, span 1) touch the
// same element set j + r N/R per butterfly, so they run in registers with a
// single shared-memory round trip.  mod(b, k, value) returns the new value
// of spectrum element k of transform b.
template <int N, int R, int NT, int BATCH, class A, class Mod>
__device__ __forceinline__ void fft_mid_pass(float2 *__restrict__ s, const float2 *__restrict__ tw,
                                             Mod &mod) {
  constexpr int NJ = N / R;
  constexpr int PER = BATCH * NJ / NT;
  static_assert(PER >= 1 && PER * NT == BATCH * NJ, "butterflies must split evenly");
  float2 v[PER][R];
  int bb[PER], jj[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int u = threadIdx.x + i * NT;
    const int j = u % NJ, b = u / NJ;
    bb[i] = b;
    jj[i] = j;
#pragma unroll
    for (int r = 0; r < R; ++r) v[i][r] = s[A::at(b, j + r * NJ)];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int j = jj[i];
#pragma unroll
    for (int r = 1; r < R; ++r) v[i][r] = cmul(v[i][r], tw[r * j]);
    dft<R, false>(v[i]);
#pragma unroll
    for (int r = 0; r < R; ++r) v[i][r] = mod(bb[i], j + r * NJ, v[i][r]);
    dft<R, true>(v[i]);
#pragma unroll
    for (int r = 0; r < R; ++r) s[A::at(bb[i], j * R + r)] = v[i][r];
  }
  __syncthreads();
}

// Full 1-D transforms along the tile's transform axis.  Radix plans:
// 64 = 8.8, 128 = 16.8, 256 = 16.16, 512 = 8.8.8.
template <int N, bool INV, int NT, int BATCH, bool JFAST, class A>
__device__ __forceinline__ void fft_all(float2 *s, const float2 *tw) {
  if constexpr (N == 64) {
    fft_pass<64, 8, 1, INV, NT, BATCH, JFAST, A>(s, tw);
    fft_pass<64, 8, 8, INV, NT, BATCH, JFAST, A>(s, tw);
  } else if constexpr (N == 128) {
    fft_pass<128, 16, 1, INV, NT, BATCH, JFAST, A>(s, tw);
    fft_pass<128, 8, 16, INV, NT, BATCH, JFAST, A>(s, tw);
  } else if constexpr (N == 256) {
    fft_pass<256, 16, 1, INV, NT, BATCH, JFAST, A>(s, tw);
    fft_pass<256, 16, 16, INV, NT, BATCH, JFAST, A>(s, tw);
  } else if constexpr (N == 512) {
    fft_pass<512, 8, 1, INV, NT, BATCH, JFAST, A>(s, tw);
    fft_pass<512, 8, 8, INV, NT, BATCH, JFAST, A>(s, tw);
    fft_pass<512, 8, 64, INV, NT, BATCH, JFAST, A>(s, tw);
  } else {
    static_assert(N == 64 || N == 128 || N == 256 || N == 512, "frame side");
  }
}

// Forward transform, pointwise map, inverse transform along rows (j fastest).
template <int N, int NT, int BATCH, class A, class Mod>
__device__ __forceinline__ void fft_roundtrip_rows(float2 *s, const float2 *tw, Mod &mod) {
  if constexpr (N == 64) {
    fft_pass<64, 8, 1, false, NT, BATCH, true, A>(s, tw);
    fft_mid_pass<64, 8, NT, BATCH, A>(s, tw, mod);
    fft_pass<64, 8, 8, true, NT, BATCH, true, A>(s, tw);
  } else if constexpr (N == 128) {
    fft_pass<128, 16, 1, false, NT, BATCH, true, A>(s, tw);
    fft_mid_pass<128, 8, NT, BATCH, A>(s, tw, mod);
    fft_pass<128, 16, 8, true, NT, BATCH, true, A>(s, tw);
  } else if constexpr (N == 256) {
    fft_pass<256, 16, 1, false, NT, BATCH, true, A>(s, tw);
    fft_mid_pass<256, 16, NT, BATCH, A>(s, tw, mod);
    fft_pass<256, 16, 16, true, NT, BATCH, true, A>(s, tw);
  } else if constexpr (N == 512) {
    fft_pass<512, 8, 1, false, NT, BATCH, true, A>(s, tw);
    fft_pass<512, 8, 8, false, NT, BATCH, true, A>(s, tw);
    fft_mid_pass<512, 8, NT, BATCH, A>(s, tw, mod);
    fft_pass<512, 8, 8, true, NT, BATCH, true, A>(s, tw);
    fft_pass<512, 8, 64, true, NT, BATCH, true, A>(s, tw);
  }
}

// ------------------------------------------------------------------ PTX: mbarrier + bulk copy

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> this CTA's shared memory, completion on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// L2 policy for data read once per sweep (the streamed frame set): evict first
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// L2 policy for data revisited by later launches (the object): evict last
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// 8-byte global load / store carrying an L2 cache policy
__device__ __forceinline__ float2 ld_l2hint(const float2 *p, uint64_t pol) {
  float2 v;
  asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
               : "=f"(v.x), "=f"(v.y)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_l2hint(float2 *p, float2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y),
               "l"(pol)
               : "memory");
}
// as bulk_g2s, with an L2 cache policy for the source
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of `bar`, giving up after `limit_ns`.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// Tensor memory (TMEM): allocation by one whole warp (a power of two >= 32
// columns), release of the allocation permit, and the fences that order
// tcgen05 operations around thread synchronisation.
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 16 consecutive 32-bit columns of this thread's TMEM lane (warp-collective:
// warp w reaches lanes 32 (w % 4) .. 32 (w % 4) + 31)
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]),
      "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]),
      "f"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
        "=f"(v[7]), "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]),
        "=f"(v[13]), "=f"(v[14]), "=f"(v[15])
      : "r"(taddr)
      : "memory");
}
// 8 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
        "=f"(v[7])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Programmatic dependent launch: wait until the preceding kernel in the
// stream has completed and its writes are visible; let the next kernel's
// CTAs start their independent prologue early.
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_dependents_launch() {
  asm volatile("griddepcontrol.launch_dependents;" :::);
}

// ------------------------------------------------------------------ reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
// the same as a butterfly: every lane ends with the (identical) sum
__device__ __forceinline__ double warp_sum_all(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// lane holding the largest q (FP32 comparison) hands its (re, im) to every lane
__device__ __forceinline__ float2 warp_argmax_f(float q, float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float q2 = __shfl_xor_sync(0xffffffffu, q, o);
    const float vx = __shfl_xor_sync(0xffffffffu, v.x, o);
    const float vy = __shfl_xor_sync(0xffffffffu, v.y, o);
    if (q2 > q) {
      q = q2;
      v = make_float2(vx, vy);
    }
  }
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// s + c += v, error-free in FP32 (Knuth's two-sum): the pair (s, c) carries
// the exact sum of the values added to about 2^-48 relative, without the
// FP64 pipe (narrow on this GPU)
__device__ __forceinline__ void two_sum_add(float &s, float &c, float v) {
  const float t = s + v, bp = t - s;
  c += (s - (t - bp)) + (v - bp);
  s = t;
}

// the value of a two-sum pair in FP64; an infinite sum stays infinite (its
// error term is NaN then)
__device__ __forceinline__ double two_sum_value(float hi, float lo) {
  return isfinite(hi) ? static_cast<double>(hi) + static_cast<double>(lo) : static_cast<double>(hi);
}

// (hi, lo) <- the warp's sum of the lanes' (hi + lo), two-sum at every level
// of the butterfly tree (lane 0's result is the one to use)
__device__ __forceinline__ void warp_two_sum(float &hi, float &lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    two_sum_add(hi, lo, h2);
    lo += l2;
  }
}

// intensity element -> float
__device__ __forceinline__ float ival(uint16_t v) { return static_cast<float>(v); }
__device__ __forceinline__ float ival(__half v) { return __half2float(v); }
__device__ __forceinline__ float ival(float v) { return v; }

}  // namespace epie
