// epie_fused_128.cu -- the fused ePIE position-update kernels for 128 x 128
// frames, in three tile shapes: 1, 2 or 4 (the default) CTAs per frame.
//
// The 1-CTA shape is its own kernel: one CTA of 1024 threads owns one scan
// position of a group (the ePIE step of Maiden & Rodenburg 2009, as the
// paper's engine runs it, Sec. "ePIE Implementation"), every thread holds 16
// complex values, and the 2-D transform runs as a radix-16 and a radix-8
// stage along each axis (128 = 16 x 8), each stage in place on the set of
// elements it reads:
//
//   forward (decimation in frequency), for n = j + 8 r (j < 8, r < 16),
//   k = k1 + 16 k2 (k1 < 16, k2 < 8):
//     stage A  thread j: Y[k1] = sum_r x[j + 8 r] W16^(r k1), times
//              W128^(j k1), stored at j + 8 k1;
//     stage B  thread jj, for k1 = 2 jj and 2 jj + 1:
//              X[k1 + 16 k2] = sum_j Y[j + 8 k1] W8^(j k2), stored at
//              8 k1 + k2 (the spectrum in digit-reversed order);
//   inverse (decimation in time) from that order back to natural order:
//     stage B' Z[j] = sum_k2 X'[8 k1 + k2] W8^(-j k2), times W128^(-j k1),
//              stored at 8 k1 + j;
//     stage A' x'[j + 8 r] = sum_k1 Z[8 k1 + j] W16^(-r k1).
//
// The whole frame's tile ([row][129] complex, the odd pitch keeps both the
// column and the row passes free of bank conflicts) and its amplitude tile
// sit in one CTA's shared memory, so the transposes between the column and
// the row passes are plain __syncthreads barriers, with no cluster and no
// distributed shared memory.  The object patch and probe values are parked
// in tensor memory for the update (all 512 columns: one CTA per SM).
// Twiddles W128^m are in constant memory; every twiddle index is
// warp-uniform.
//
// The 2- and 4-CTA shapes are the general kernel of epie_fused.cuh; they
// read the amplitudes in plain FFT order.  Spreading a frame over 4 SMs
// shortens the step of a small colour class (tens of frames), so 4 is the
// default; one CTA per frame suits large groups (mini-batches of hundreds).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "epie_fused.cuh"
#include "epie_ingest.cuh"

namespace epie {

namespace {

constexpr int S_N = 128, S_NT = 1024, S_NW = 32;
constexpr int TP = 129;                      // tile pitch (complex)
constexpr int TILE = S_N * TP;
constexpr size_t OFF_AMP = sizeof(float2) * TILE;
constexpr uint32_t AMP_BYTES = S_N * S_N * sizeof(float);  // the frame's amplitude tile
constexpr size_t STAGE_BYTES = S_N * (S_N * 4 + 16);       // raw rows of any type, padded
constexpr size_t OFF_RED = OFF_AMP + STAGE_BYTES;          // float4 per warp
constexpr size_t OFF_CAND = OFF_RED + 16 * S_NW;           // float4 per warp
constexpr size_t OFF_BAR = OFF_CAND + 16 * S_NW;
constexpr size_t SMEM128 = OFF_BAR + 16;  // mbarrier, then the TMEM address slot
constexpr int TM_COLS = 512;              // 64 columns per thread, 8 warps per lane quadrant
static_assert(AMP_BYTES <= STAGE_BYTES, "the amplitude tile fits the staging area");
static_assert(OFF_AMP % 16 == 0 && OFF_RED % 16 == 0 && OFF_CAND % 16 == 0 && OFF_BAR % 8 == 0,
              "alignment of the shared-memory regions");
static_assert(SMEM128 <= 227 * 1024, "one CTA's shared memory");

// raw intensity rows (allocation-free entry point): 128 rows of 128 values,
// row pitch a multiple of 16 bytes (bulk-copy destinations)
template <typename IT>
struct RawRows {
  static constexpr int PITCH = S_N * static_cast<int>(sizeof(IT)) + 16;
  static_assert(S_N * PITCH <= static_cast<int>(STAGE_BYTES), "raw rows fit the staging area");
};

__constant__ float2 c_tw128[S_N];  // exp(-2 pi i m / 128)

// spectrum position p of the digit-reversed order holds frequency
// (p >> 3) + 16 (p & 7)
__device__ __forceinline__ int freq_of_pos(int p) { return (p >> 3) + 16 * (p & 7); }

template <bool INV>
__device__ __forceinline__ float2 tw128(int m) {
  float2 w = c_tw128[m];
  if (INV) w.y = -w.y;
  return w;
}

// the two radix-8 DFTs of a thread's halves v[0..8) and v[8..16)
template <bool INV>
__device__ __forceinline__ void dft8_pair(float2 (&v)[16]) {
  float2 lo[8], hi[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    lo[i] = v[i];
    hi[i] = v[8 + i];
  }
  dft8<INV>(lo);
  dft8<INV>(hi);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    v[i] = lo[i];
    v[8 + i] = hi[i];
  }
}

template <typename IT, bool MB>
__global__ void __launch_bounds__(S_NT, 1) epie_fused128_kernel(GroupArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  float2 *tile = reinterpret_cast<float2 *>(smem);
  float *ampt = reinterpret_cast<float *>(smem + OFF_AMP);
  float4 *red = reinterpret_cast<float4 *>(smem + OFF_RED);
  float4 *cand = reinterpret_cast<float4 *>(smem + OFF_CAND);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + OFF_BAR);
  uint32_t *tm_slot = reinterpret_cast<uint32_t *>(smem + OFF_BAR + 8);

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int member = blockIdx.x;
  const int32_t *members = a.members;
  int n_members = a.n_members;
  if (a.gstart) {
    // device group table: a CTA past the group's size exits here, before any
    // barrier or copy
    const int g0 = a.gstart[a.group];
    n_members = a.gstart[a.group + 1] - g0;
    if (member >= n_members) return;
    members += g0;
  }
  const int f = members[member];
  const int py = a.pos[2 * f], px = a.pos[2 * f + 1];
  // (failure injection: the launch's first CTA never issues its copies)
  const bool issue = !(a.inject_skip_copy && blockIdx.x == 0);
  unsigned char *raw = smem + OFF_AMP;

  if (w == 0) tmem_alloc(tm_slot, TM_COLS);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    if (issue) {
      if (a.amp) {
        // the frame's amplitude tile, read once per sweep: keep it from
        // evicting the object
        mbar_arrive_expect_tx(bar, AMP_BYTES);
        bulk_g2s_hint(ampt, a.amp + static_cast<size_t>(f) * S_N * S_N, AMP_BYTES, bar,
                      l2_evict_first_policy());
      } else {
        mbar_arrive_expect_tx(bar, static_cast<uint32_t>(S_N * S_N * sizeof(IT)));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (!a.amp && tid < S_N && issue) {
    // raw intensities: frequency row ky(p) into staging row p
    const IT *frame = static_cast<const IT *>(a.frames) + static_cast<size_t>(f) * S_N * S_N;
    bulk_g2s_hint(raw + tid * RawRows<IT>::PITCH, frame + freq_of_pos(tid) * S_N, S_N * sizeof(IT), bar,
                  l2_evict_first_policy());
  }
  // this thread's tensor-memory columns: [0, 32) object patch, [32, 64) probe
  const uint32_t tm = *tm_slot + (static_cast<uint32_t>(32 * (w & 3)) << 16) +
                      static_cast<uint32_t>((w >> 2) * 64);
  const uint64_t wait_ns = a.wait_ns ? a.wait_ns : 2000000000ull;

  // ---------------------------------------------------------------- columns
  // thread (x = 32 (w & 3) + lane, j = w >> 2): elements y = j + 8 r
  const int x = 32 * (w & 3) + lane, j = w >> 2;
  const size_t orow = static_cast<size_t>(a.W);
  float2 *Ob = a.O + static_cast<size_t>(py + j) * orow + px + x;
  const float2 *Pb = a.P + j * S_N + x;
  const uint64_t opol = l2_evict_last_policy();  // the object is revisited by later classes
  float2 v[16];
  float om = -1.f;
  float2 omv = make_float2(0.f, 0.f);
  // The object patch is read before the dependency wait when o_early says it
  // is final; the probe, max|P|^2 and the partial buffers are written by the
  // preceding kernels and are read after it.
  if (!a.o_early) grid_dependency_wait();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = ld_l2hint(Ob + static_cast<size_t>(8 * r) * orow, opol);
  if (a.o_early) grid_dependency_wait();
  grid_dependents_launch();
  if (blockIdx.x == 0 && tid == 0 && a.pmax2_clear) *a.pmax2_clear = 0ull;
  double pm = 0.0;
  if (tid == 0) pm = __longlong_as_double(static_cast<long long>(*a.pmax2));
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float keep[16];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 o = v[8 * h + i];
      const float q = o.x * o.x + o.y * o.y;
      if (q > om) {
        om = q;
        omv = o;
      }
      keep[2 * i] = o.x;
      keep[2 * i + 1] = o.y;
    }
    tmem_st16(tm + 16 * h, keep);
  }
  // the probe in one round trip; the exit wave multiplies the parked object
  // values back in
  tmem_wait_st();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = __ldg(Pb + r * 8 * S_N);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float keep[16];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      keep[2 * i] = v[8 * h + i].x;
      keep[2 * i + 1] = v[8 * h + i].y;
    }
    tmem_st16(tm + 32 + 16 * h, keep);
  }
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    float ko[8];
    tmem_ld8(tm + 8 * h, ko);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 4; ++i) v[4 * h + i] = cmul(v[4 * h + i], make_float2(ko[2 * i], ko[2 * i + 1]));
  }
  // column stage A
  dft16<false>(v);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], tw128<false>(j * k1));
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) tile[(j + 8 * k1) * TP + x] = v[k1];
  // max |O_old|^2 over the patch: FP32 comparisons pick the element, its
  // square is formed in FP64
  omv = warp_argmax_f(om, omv);
  if (lane == 0) cand[w] = make_float4(omv.x, omv.y, omv.x * omv.x + omv.y * omv.y, 0.f);
  tmem_wait_st();
  __syncthreads();
  // column stage B: k1 = 2 j (v[0..8)) and 2 j + 1 (v[8..16)), rows 16 j + ..
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = tile[(16 * j + i) * TP + x];
  dft8_pair<false>(v);
#pragma unroll
  for (int i = 0; i < 16; ++i) tile[(16 * j + i) * TP + x] = v[i];
  if (w == 0) {
    // max|O_old|^2 of the patch, then the update strengths alpha / max|P|^2
    // and beta / max|O_old|^2 (FP64 maxima, FP32 divisions), read by every
    // thread after the next barrier
    const float4 cd = cand[lane];
    const float2 cv = warp_argmax_f(cd.z, make_float2(cd.x, cd.y));
    if (lane == 0) {
      const double omp = static_cast<double>(cv.x) * cv.x + static_cast<double>(cv.y) * cv.y;
      const double om_used = a.omax2_global ? *a.omax2_global : omp;
      float *st = reinterpret_cast<float *>(smem + OFF_CAND);  // the candidates are consumed
      const float pmf = static_cast<float>(pm), omf = static_cast<float>(om_used);
      st[0] = pm > 0.0 ? a.alpha / pmf : 0.f;
      st[1] = om_used > 0.0 ? a.beta / omf : 0.f;
      st[2] = pm > 0.0 ? 1.0f / pmf : 0.f;
    }
  }
  __syncthreads();

  // ---------------------------------------------------------------- rows
  // thread (p = 32 (w & 3) + lane, j = w >> 2): spectrum row p, x = j + 8 r
  const int p = x;
  // row stage A
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = tile[p * TP + j + 8 * r];
  dft16<false>(v);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], tw128<false>(j * k1));
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) tile[p * TP + j + 8 * k1] = v[k1];
  bool ok = mbar_wait_bounded(bar, 0, wait_ns);
  if (!ok) atomicOr(a.err_flag, FLAG_TMA_TIMEOUT);
  ok = __all_sync(0xffffffffu, ok);  // warp-uniform: the update reads TMEM warp-collectively
  float isum_s = 0.f, isum_c = 0.f;  // sum I of this thread's converted values (raw path)
  if (!a.amp) {
    // raw rows -> sqrt(max(I - dark, 0)) in the amplitude layout, in place:
    // every raw value is read before the barrier, every float written after
    float iv[16];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int ci = tid + S_NT * u, pr = ci & 127, jm = ci >> 7;
      const int kx0 = 2 * (jm >> 2) + ((jm & 3) >> 1) + 64 * (jm & 1);
      const IT *row = reinterpret_cast<const IT *>(raw + pr * RawRows<IT>::PITCH);
#pragma unroll
      for (int i = 0; i < 4; ++i) iv[4 * u + i] = ival(row[kx0 + 16 * i]);
      if (a.dark) {
        const float *drow = a.dark + freq_of_pos(pr) * S_N;
#pragma unroll
        for (int i = 0; i < 4; ++i) iv[4 * u + i] -= __ldg(drow + kx0 + 16 * i);
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float4 o;
      float *op = &o.x;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float I = fmaxf(iv[4 * u + i], 0.f);  // also maps NaN to 0
        two_sum_add(isum_s, isum_c, I);
        op[i] = sqrtf(I);
      }
      reinterpret_cast<float4 *>(ampt)[tid + S_NT * u] = o;
    }
  }
  __syncthreads();
  // row stage B, modulus replacement, row stage B': k1 = 2 j (v[0..8)) and
  // 2 j + 1 (v[8..16))
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = tile[p * TP + 16 * j + i];
  dft8_pair<false>(v);
  float e = 0.f;
  {
    // chunk (j * 4 + m) * 128 + p holds the amplitudes of k1 = 2 j + (m >> 1),
    // k2 = 4 (m & 1) + i: element 4 m + i of v
    const float4 *a4 = reinterpret_cast<const float4 *>(ampt) + j * 4 * 128 + p;
    constexpr float invK = 1.0f / (float(S_N) * float(S_N));
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const float4 s4 = a4[128 * m];
      const float sq[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float2 &z = v[4 * m + i];
        const float a2 = z.x * z.x + z.y * z.y;
        float amp;
        if (a2 > 0.f) {
          const float ia = rsqrtf(a2);
          amp = a2 * ia;
          const float rr = sq[i] * ia * invK;
          z = __fmul2_rn(z, make_float2(rr, rr));  // both components, one instruction
        } else {
          amp = 0.f;
          z = make_float2(sq[i] * invK, 0.f);
        }
        const float d = amp - sq[i];
        e = fmaf(d, d, e);
      }
    }
  }
  dft8_pair<true>(v);
#pragma unroll
  for (int i = 1; i < 8; ++i) {
    v[i] = cmul(v[i], tw128<true>(i * 2 * j));
    v[8 + i] = cmul(v[8 + i], tw128<true>(i * (2 * j + 1)));
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) tile[p * TP + 16 * j + i] = v[i];
  {
    // error terms: FP32 over a thread's 16 elements, then an error-free
    // (two-sum) FP32 tree over the warp; FP64 only across warps, in one warp
    float eh = e, el = 0.f, sh = isum_s, sl = isum_c;
    warp_two_sum(eh, el);
    warp_two_sum(sh, sl);
    if (lane == 0) red[w] = make_float4(eh, el, sh, sl);
  }
  __syncthreads();
  // row stage A': x = j + 8 r
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) v[k1] = tile[p * TP + 8 * k1 + j];
  dft16<true>(v);
#pragma unroll
  for (int r = 0; r < 16; ++r) tile[p * TP + j + 8 * r] = v[r];
  __syncthreads();
  if (w == 0) {
    const float4 t = red[lane];
    double es = two_sum_value(t.x, t.y), ss = two_sum_value(t.z, t.w);
    es = warp_sum_all(es);
    ss = warp_sum_all(ss);
    if (lane == 0) {
      a.err_part[static_cast<size_t>(f) * a.err_stride] = es;
      a.isum_part[static_cast<size_t>(f) * a.err_stride] = a.amp ? a.amp_isum[f] : ss;
    }
  }

  // ---------------------------------------------------------------- columns, inverse
  // column stage B': k1 = 2 j (v[0..8)) and 2 j + 1 (v[8..16)), rows 16 j + ..
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = tile[(16 * j + i) * TP + x];
  dft8_pair<true>(v);
#pragma unroll
  for (int i = 1; i < 8; ++i) {
    v[i] = cmul(v[i], tw128<true>(i * 2 * j));
    v[8 + i] = cmul(v[8 + i], tw128<true>(i * (2 * j + 1)));
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) tile[(16 * j + i) * TP + x] = v[i];
  __syncthreads();
  // column stage A' -> psi' at y = j + 8 r
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) v[k1] = tile[(8 * k1 + j) * TP + x];
  dft16<true>(v);

  const float *st = reinterpret_cast<const float *>(smem + OFF_CAND);  // written before the barriers
  const float ao = st[0], bp = st[1];
  float2 *part = a.probe_part + static_cast<size_t>(member) * S_N * S_N + j * S_N + x;
  if (ok) {
    if constexpr (!MB) {
      // the per-element scalings as paired-FP32 operations (each lane rounds
      // as the scalar fmaf / multiply would)
      const float2 ao2 = make_float2(ao, ao), bp2 = make_float2(bp, bp);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float ko[8], kp[8];
        tmem_ld8(tm + 8 * h, ko);
        tmem_ld8(tm + 32 + 8 * h, kp);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = 4 * h + i;
          const float2 o = make_float2(ko[2 * i], ko[2 * i + 1]);
          const float2 pp = make_float2(kp[2 * i], kp[2 * i + 1]);
          const float2 d = psub(v[r], cmul(pp, o));
          const float2 uo = cmulc(pp, d);  // conj(P) Delta
          const float2 up = cmulc(o, d);   // conj(O_old) Delta
          st_l2hint(Ob + static_cast<size_t>(8 * r) * orow, __ffma2_rn(ao2, uo, o), opol);
          part[8 * r * S_N] = __fmul2_rn(up, bp2);
        }
      }
    } else {
      // mini-batch: patches of a batch may overlap; the object moves once per
      // batch by the count-normalised sum, applied by a separate kernel
      const float inv_pm = st[2];
      const size_t obase = static_cast<size_t>(py + j) * orow + px + x;
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float ko[8], kp[8];
        tmem_ld8(tm + 8 * h, ko);
        tmem_ld8(tm + 32 + 8 * h, kp);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = 4 * h + i;
          const float2 o = make_float2(ko[2 * i], ko[2 * i + 1]);
          const float2 pp = make_float2(kp[2 * i], kp[2 * i + 1]);
          const float2 d = csub(v[r], cmul(pp, o));
          const float2 uo = cscale(cmulc(pp, d), inv_pm);
          const size_t oi = obase + static_cast<size_t>(8 * r) * orow;
          atomicAdd(a.accO + oi, uo);  // one paired (8-byte) atomic
          atomicAdd(a.cnt + oi, 1);
          part[8 * r * S_N] = cscale(cmulc(o, d), bp);
        }
      }
    }
  } else {
    // the copy never arrived: give it one more bounded wait before exiting
    mbar_wait_bounded(bar, 0, wait_ns < 100000000ull ? wait_ns : 100000000ull);
  }
  // every thread's tensor-memory reads are done before warp 0 frees it
  tc_fence_before();
  __syncthreads();
  if (w == 0) {
    tc_fence_after();
    tmem_dealloc(*tm_slot, TM_COLS);
  }
}

// Measured amplitudes of frames [f0, f0 + n) in the layout of the 1-CTA step
// kernel's amplitude tile: float4 chunk (jj * 4 + m) * 128 + p holds, for
// spectrum row p (frequency ky = (p >> 3) + 16 (p & 7)), the values at
// kx = k1 + 16 (4 (m & 1) + i), k1 = 2 jj + (m >> 1), i = 0..3.
// amp = sqrt(max(I - dark, 0)); isum = sum of max(I - dark, 0), two-sum in
// FP32 per thread and a fixed-order FP64 sum over the block.  One block per
// frame: each thread loads its chunks of the 128 rows (four 32-row tiles) as
// 16-byte vectors, all in flight at once (TileLane), into shared memory; the
// block then writes the frame chunk by chunk (coalesced).
constexpr int AI_NT = 512, AI_PITCH = S_N + 1;  // odd pitch: conflict-free chunk reads
constexpr size_t AI_SMEM = sizeof(float) * S_N * AI_PITCH + sizeof(double) * AI_NT;
template <typename IT>
__global__ void __launch_bounds__(AI_NT) amp_ingest128_kernel(const IT *__restrict__ frames,
                                                              const float *__restrict__ dark,
                                                              float *__restrict__ amp,
                                                              double *__restrict__ isum, int f0) {
  extern __shared__ __align__(16) unsigned char ai_smem[];
  float *rows = reinterpret_cast<float *>(ai_smem);
  double *sh = reinterpret_cast<double *>(ai_smem + sizeof(float) * S_N * AI_PITCH);
  const size_t fb = static_cast<size_t>(f0 + blockIdx.x) * S_N * S_N;
  const IT *fr = frames + fb;
  float4 *out = reinterpret_cast<float4 *>(amp + fb);
  const int t = threadIdx.x;
  float s = 0.f, cc = 0.f;
  TileLane<S_N, AI_NT, IT> tl[S_N / 32];
#pragma unroll
  for (int q = 0; q < S_N / 32; ++q) tl[q].load(fr, freq_of_pos(32 * q + tl[q].yl));
#pragma unroll
  for (int q = 0; q < S_N / 32; ++q)
    tl[q].store(rows + 32 * q * AI_PITCH, dark, freq_of_pos(32 * q + tl[q].yl), s, cc);
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4096 / AI_NT; ++u) {
    const int ci = t + AI_NT * u, pr = ci & 127, jm = ci >> 7;
    const int kx0 = 2 * (jm >> 2) + ((jm & 3) >> 1) + 64 * (jm & 1);
    const float *r = rows + pr * AI_PITCH + kx0;
    out[ci] = make_float4(r[0], r[16], r[32], r[48]);
  }
  sh[t] = two_sum_value(s, cc);
  __syncthreads();
  for (int h = AI_NT / 2; h > 0; h >>= 1) {
    if (t < h) sh[t] += sh[t + h];
    __syncthreads();
  }
  if (t == 0) isum[f0 + blockIdx.x] = sh[0];
}

bool g_tw_ready[64] = {};

template <typename IT, bool MB>
cudaError_t launch_one(const GroupArgs &a, cudaStream_t st) {
  auto kern = epie_fused128_kernel<IT, MB>;
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_tw_ready[dev]) {
    // twiddles exp(-2 pi i m / 128), evaluated in double precision
    float2 tw[S_N];
    for (int m = 0; m < S_N; ++m) {
      const double ang = -2.0 * 3.14159265358979323846 * m / S_N;
      tw[m] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
    }
    cudaError_t e = cudaMemcpyToSymbol(c_tw128, tw, sizeof tw);
    if (e != cudaSuccess) return e;
    g_tw_ready[dev] = true;
  }
  if (!configured[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(SMEM128));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    // A TMEM allocation blocks until columns are free: every CTA that can be
    // resident on an SM must find its 512 columns at once (one resident CTA)
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, S_NT, SMEM128);
    if (e != cudaSuccess) return e;
    if (occ != 1) return cudaErrorInvalidConfiguration;
    configured[dev] = true;
  }
  if (a.n_members <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(a.n_members), 1, 1);
  cfg.blockDim = dim3(S_NT, 1, 1);
  cfg.dynamicSmemBytes = SMEM128;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

// the 2- and 4-CTA shapes: the general kernel (epie_fused.cuh)
template <int CL>
cudaError_t launch_cl(int itype, const GroupArgs &a, cudaStream_t st) {
  constexpr int NT = 128 * 128 / (CL * 16);
  if (itype == 0) return launch_fused_t<128, CL, NT, uint16_t>(a, st);
  if (itype == 1) return launch_fused_t<128, CL, NT, __half>(a, st);
  return launch_fused_t<128, CL, NT, float>(a, st);
}

template <typename IT>
cudaError_t amp_ingest_t(const IT *frames, const float *dark, float *amp, double *isum, int f0, int n,
                         cudaStream_t st) {
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!configured[dev]) {
    cudaError_t e = cudaFuncSetAttribute(amp_ingest128_kernel<IT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(AI_SMEM));
    if (e != cudaSuccess) return e;
    configured[dev] = true;
  }
  amp_ingest128_kernel<IT><<<n, AI_NT, AI_SMEM, st>>>(frames, dark, amp, isum, f0);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fused_128(int itype, const GroupArgs &a, cudaStream_t st, int cl) {
  switch (cl == 0 ? EPIE_CTAS_128 : cl) {
    case 1: {
      // the mini-batch update (object-update accumulator) is its own instantiation
      const bool mb = a.accO != nullptr;
      if (itype == 0) return mb ? launch_one<uint16_t, true>(a, st) : launch_one<uint16_t, false>(a, st);
      if (itype == 1) return mb ? launch_one<__half, true>(a, st) : launch_one<__half, false>(a, st);
      return mb ? launch_one<float, true>(a, st) : launch_one<float, false>(a, st);
    }
    case 2: return launch_cl<2>(itype, a, st);
    case 4: return launch_cl<4>(itype, a, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t fused_smem_128(int itype) {
  // the default shape's shared memory (EPIE_CTAS_128 CTAs per frame)
  constexpr int CL = EPIE_CTAS_128;
  if constexpr (CL == 1) {
    return SMEM128;
  } else {
    constexpr int NT = 128 * 128 / (CL * 16);
    if (itype == 0) return FusedCfg<128, CL, NT, uint16_t>::SMEM;
    if (itype == 1) return FusedCfg<128, CL, NT, __half>::SMEM;
    return FusedCfg<128, CL, NT, float>::SMEM;
  }
}

cudaError_t launch_amp_ingest_128(const void *frames, int itype, const float *dark, float *amp,
                                  double *isum, int f0, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (itype == 0) return amp_ingest_t(static_cast<const uint16_t *>(frames), dark, amp, isum, f0, n, st);
  if (itype == 1) return amp_ingest_t(static_cast<const __half *>(frames), dark, amp, isum, f0, n, st);
  return amp_ingest_t(static_cast<const float *>(frames), dark, amp, isum, f0, n, st);
}

}  // namespace epie
