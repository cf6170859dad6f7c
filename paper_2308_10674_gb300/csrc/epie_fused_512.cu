// epie_fused_512.cu -- the fused ePIE position-update kernel for 512 x 512
// frames, and the measured-amplitude layout it reads.
//
// One thread-block cluster of 16 CTAs x 512 threads owns one scan position of
// a group (the ePIE step of Maiden & Rodenburg 2009, as the paper's engine
// runs it, Sec. "ePIE Implementation").  Each thread holds 32 complex values
// (lo = elements 0..15, hi = 16..31).  The 2-D transform runs as a radix-32
// and a radix-16 stage along each axis (512 = 32 x 16), written so that every
// stage reads and writes the same set of elements of each thread:
//
//   forward (decimation in frequency), for n = j + 16 r (j < 16, r < 32),
//   k = k1 + 32 k2 (k1 < 32, k2 < 16):
//     stage A  thread j: Y[k1] = sum_r x[j + 16 r] W32^(r k1), times
//              W512^(j k1), stored at j + 16 k1;
//     stage B  thread w, for k1 = 2w and 2w + 1:
//              X[k1 + 32 k2] = sum_j Y[j + 16 k1] W16^(j k2), stored at
//              16 k1 + k2 (the spectrum in digit-reversed order);
//   inverse (decimation in time) from that order back to natural order:
//     stage B' thread w, k1 = 2w, 2w + 1: Z[j] = sum_k2 X'[16 k1 + k2]
//              W16^(-j k2), times W512^(-j k1), stored at 16 k1 + j;
//     stage A' thread j: x'[j + 16 r] = sum_k1 Z[16 k1 + j] W32^(-r k1).
//
//   phase 1  CTA c, columns [32c, 32c + 32): each thread loads the object
//            patch and probe of its 32 elements (x = 32c + lane,
//            y = w + 16 r, w = warp) into registers, parks them in tensor
//            memory, forms psi = P . O_j and runs column stage A; then
//            column stage B and a push of the finished column spectra into
//            the peer CTA that owns their row block (st.shared::cluster,
//            between split cluster barriers);
//   phase 2  CTA q, row positions [32q, 32q + 32): row stages A and B, the
//            modulus replacement with sqrt(I) (the amplitude tile, in the
//            order of the digit-reversed spectrum, arrives by one bulk copy
//            issued at kernel start) and row stage B', then row stage A' and
//            a push of the rows back to the column owners;
//   phase 3  column stages B' and A' give psi' for exactly the 32 elements
//            each thread loaded in phase 1: Delta, the object update and the
//            probe-update partial are formed in registers, with O_old and P
//            read back from tensor memory.
//
// Shared memory holds the CTA's tile (phase 1 [row position][33], phase 2
// [row][513], phase 3 [column][513] complex: odd pitches keep every stage
// free of bank conflicts, and both pushes write runs of 32 consecutive
// elements per warp), the amplitude tile and a few reduction slots: one CTA
// per SM, which also owns all 512 tensor-memory columns.  Twiddles W512^m are
// in constant memory; every twiddle index is warp-uniform.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "epie_cluster.cuh"
#include "epie_fft.cuh"
#include "epie_ingest.cuh"
#include "epie_internal.h"

namespace epie {

namespace {

constexpr int S_N = 512, S_CL = 16, S_NT = 512, S_NW = 16;
// clusters (frames) one wave of this kernel holds on a GB300 (one CTA per
// SM, a 16-CTA cluster per GPC): a hint for the second-wave L2 prefetch only
constexpr int S_WAVE = 9;
static_assert(EPIE_CTAS_512 == S_CL, "the 512^2 kernel runs 16-CTA clusters");
constexpr int CP = 33;                       // column-tile pitch (complex)
constexpr int RP = 513;                      // row-tile pitch (complex)
constexpr int CT = 513;                      // phase-3 tile: [column][row position]
constexpr int SLAB = S_N * CP;               // >= 32 * RP
constexpr size_t OFF_AMP = sizeof(float2) * SLAB;
constexpr uint32_t AMP_BYTES = 32 * S_N * sizeof(float);  // one CTA's amplitude tile
constexpr size_t STAGE_BYTES = 32 * (S_N * 4 + 16);       // raw rows of any type, padded
constexpr size_t OFF_RED = OFF_AMP + STAGE_BYTES;         // float4 per warp
constexpr size_t OFF_OMAX = OFF_RED + 16 * S_NW;          // 16 cluster slots (double)
constexpr size_t OFF_CAND = OFF_OMAX + sizeof(double) * S_CL;  // float4 per warp
constexpr size_t OFF_BAR = OFF_CAND + 16 * S_NW;
constexpr size_t SMEM512 = OFF_BAR + 16;  // mbarrier, then the TMEM address slot
constexpr int TM_COLS = 512;              // 128 columns per thread, 4 warps per lane quadrant
static_assert(32 * RP <= SLAB && 32 * CT <= SLAB, "row and phase-3 tiles fit the slab");
static_assert(AMP_BYTES <= STAGE_BYTES, "the amplitude tile fits the staging area");
static_assert(OFF_AMP % 16 == 0 && OFF_RED % 16 == 0 && OFF_CAND % 16 == 0 && OFF_BAR % 8 == 0,
              "alignment of the shared-memory regions");
static_assert(SMEM512 <= 227 * 1024, "one CTA's shared memory");

// raw intensity rows (allocation-free entry point): 32 rows of 512 values,
// row pitch a multiple of 16 bytes (bulk-copy destinations)
template <typename IT>
struct RawRows {
  static constexpr int PITCH = S_N * static_cast<int>(sizeof(IT)) + 16;
  static_assert(32 * PITCH <= static_cast<int>(STAGE_BYTES), "raw rows fit the staging area");
};

__constant__ float2 c_tw512[S_N];  // exp(-2 pi i m / 512)

// row position p of the digit-reversed spectrum holds frequency
// (p >> 4) + 32 (p & 15)
__device__ __forceinline__ int freq_of_pos(int p) { return (p >> 4) + 32 * (p & 15); }

template <bool INV>
__device__ __forceinline__ float2 tw512(int m) {
  float2 w = c_tw512[m];
  if (INV) w.y = -w.y;
  return w;
}

// element e of a thread's (lo, hi) pair of 16-element arrays
#define EL(e) ((e) < 16 ? lo[(e)] : hi[(e) - 16])

template <typename IT, bool MB>
__global__ void __launch_bounds__(S_NT, 1) epie_fused512_kernel(GroupArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  float2 *slab = reinterpret_cast<float2 *>(smem);
  float *ampt = reinterpret_cast<float *>(smem + OFF_AMP);
  float4 *red = reinterpret_cast<float4 *>(smem + OFF_RED);
  double *oslot = reinterpret_cast<double *>(smem + OFF_OMAX);
  float4 *cand = reinterpret_cast<float4 *>(smem + OFF_CAND);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + OFF_BAR);
  uint32_t *tm_slot = reinterpret_cast<uint32_t *>(smem + OFF_BAR + 8);

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int member = blockIdx.x / S_CL;
  const int32_t *members = a.members;
  int n_members = a.n_members;
  if (a.gstart) {
    // device group table: a whole cluster past the group's size exits here,
    // before any barrier or copy
    const int g0 = a.gstart[a.group];
    n_members = a.gstart[a.group + 1] - g0;
    if (member >= n_members) return;
    members += g0;
  }
  const int c = static_cast<int>(cluster_rank());
  const int f = members[member];
  const int py = a.pos[2 * f], px = a.pos[2 * f + 1];

  if (w == 0) tmem_alloc(tm_slot, TM_COLS);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // this thread's tensor-memory columns: [0, 64) object patch, [64, 128) probe
  const uint32_t tm = *tm_slot + (static_cast<uint32_t>(32 * (w & 3)) << 16) +
                      static_cast<uint32_t>((w >> 2) * 128);
  const uint64_t wait_ns = a.wait_ns ? a.wait_ns : 2000000000ull;
  // (failure injection: the launch's first CTA never issues its copies)
  const bool issue = !(a.inject_skip_copy && blockIdx.x == 0);
  unsigned char *raw = smem + OFF_AMP;
  if (a.amp) {
    // the CTA's amplitude tile, read once per sweep: keep it from evicting
    // the object
    if (tid == 0 && issue) {
      mbar_arrive_expect_tx(bar, AMP_BYTES);
      bulk_g2s_hint(ampt, a.amp + static_cast<size_t>(f) * S_N * S_N + static_cast<size_t>(c) * 32 * S_N,
                    AMP_BYTES, bar, l2_evict_first_policy());
    }
  } else if (w == 0) {
    // raw intensities: the 32 frequency rows of this CTA's row positions
    if (lane == 0 && issue) mbar_arrive_expect_tx(bar, 32u * S_N * sizeof(IT));
    __syncwarp();
    if (issue) {
      const IT *frame = static_cast<const IT *>(a.frames) + static_cast<size_t>(f) * S_N * S_N;
      const int ky = freq_of_pos(32 * c + lane);
      bulk_g2s_hint(raw + lane * RawRows<IT>::PITCH, frame + ky * S_N, S_N * sizeof(IT), bar,
                    l2_evict_first_policy());
    }
  }

  // ---------------------------------------------------------------- phase 1
  // thread (b = lane, j = w): elements y = w + 16 r, x = 32 c + lane
  const size_t orow = static_cast<size_t>(a.W);
  float2 *Ob = a.O + static_cast<size_t>(py + w) * orow + px + 32 * c + lane;
  const float2 *Pb = a.P + w * S_N + 32 * c + lane;
  const uint64_t opol = l2_evict_last_policy();  // the object is revisited by later classes
  float2 lo[16], hi[16];
  float om = -1.f;
  float2 omv = make_float2(0.f, 0.f);
  // A group larger than one wave of clusters runs a second wave: warm L2 with
  // the object rows of the frame that will take this cluster's place there
  // (a hint only; a prefetch of lines still being written is harmless).
  if (member + S_WAVE < n_members) {
    const int f2 = members[member + S_WAVE];
    const float2 *row = a.O + static_cast<size_t>(a.pos[2 * f2] + tid) * a.W + a.pos[2 * f2 + 1] + 32 * c;
    // the 16-byte-aligned interior of the 256-byte row segment (never past it)
    const uintptr_t b0 = (reinterpret_cast<uintptr_t>(row) + 15) & ~static_cast<uintptr_t>(15);
    const uintptr_t b1 = (reinterpret_cast<uintptr_t>(row + 32)) & ~static_cast<uintptr_t>(15);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b0), "r"(static_cast<uint32_t>(b1 - b0))
                 : "memory");
  }
  // The object patch is read before the dependency wait when o_early says it
  // is final; the probe, max|P|^2 and the partial buffers are written by the
  // preceding kernels and are read after it.
  if (!a.o_early) grid_dependency_wait();
#pragma unroll
  for (int r = 0; r < 32; ++r) EL(r) = ld_l2hint(Ob + static_cast<size_t>(16 * r) * orow, opol);
  if (a.o_early) grid_dependency_wait();
  grid_dependents_launch();
  if (blockIdx.x == 0 && tid == 0 && a.pmax2_clear) *a.pmax2_clear = 0ull;
  // max|P|^2 of the group (written by the preceding reduction), fetched
  // early: the update strengths are formed after the first transpose
  double pm = 0.0;
  if (tid == 0) pm = __longlong_as_double(static_cast<long long>(*a.pmax2));
  // patch maximum and the object values parked for phase 3
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    float keep[16];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 o = EL(8 * h + i);
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
  // the probe: with the object values parked, (lo, hi) take all 32 probe
  // values in one round trip; the exit wave multiplies the parked object
  // values back in
  tmem_wait_st();
#pragma unroll
  for (int r = 0; r < 32; ++r) EL(r) = __ldg(Pb + r * 16 * S_N);
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    float keep[16];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      keep[2 * i] = EL(8 * h + i).x;
      keep[2 * i + 1] = EL(8 * h + i).y;
    }
    tmem_st16(tm + 64 + 16 * h, keep);
  }
#pragma unroll
  for (int h = 0; h < 8; ++h) {
    float ko[8];
    tmem_ld8(tm + 8 * h, ko);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 4; ++i) EL(4 * h + i) = cmul(EL(4 * h + i), make_float2(ko[2 * i], ko[2 * i + 1]));
  }
  // column stage A
  dft32<false>(lo, hi);
#pragma unroll
  for (int k1 = 1; k1 < 32; ++k1) EL(k1) = cmul(EL(k1), tw512<false>(w * k1));
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) slab[(w + 16 * k1) * CP + lane] = EL(k1);
  // max |O_old|^2 over the patch: FP32 comparisons pick the element (lanes,
  // warps, then CTAs); its square is formed in FP64
  omv = warp_argmax_f(om, omv);
  if (lane == 0) cand[w] = make_float4(omv.x, omv.y, omv.x * omv.x + omv.y * omv.y, 0.f);
  tmem_wait_st();
  __syncthreads();
  // column stage B: thread (b = lane), k1 = 2 w (lo) and 2 w + 1 (hi)
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    lo[j] = slab[(32 * w + j) * CP + lane];
    hi[j] = slab[(32 * w + 16 + j) * CP + lane];
  }
  cluster_arrive();  // this CTA's tile is free once every thread has its inputs
  dft16<false>(lo);
  dft16<false>(hi);
  double om_cta = 0.0;
  if (w == 0) {
    float4 cd = lane < S_NW ? cand[lane] : make_float4(0.f, 0.f, -1.f, 0.f);
    const float2 cv = warp_argmax_f(cd.z, make_float2(cd.x, cd.y));
    om_cta = static_cast<double>(cv.x) * cv.x + static_cast<double>(cv.y) * cv.y;
  }
  cluster_wait();
  {
    // spectrum rows p = 16 k1 + k2 go to CTA k1 / 2 = w, local row
    // 16 (k1 & 1) + k2
    const uint32_t base = map_rank(smem_u32(slab), static_cast<uint32_t>(w)) +
                          8u * static_cast<uint32_t>(32 * c + lane);
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
      st_cluster(base + 8u * static_cast<uint32_t>(k2 * RP), lo[k2]);
      st_cluster(base + 8u * static_cast<uint32_t>((16 + k2) * RP), hi[k2]);
    }
    if (w == 0 && lane < S_CL)
      st_cluster(map_rank(smem_u32(oslot + c), static_cast<uint32_t>(lane)), om_cta);
  }
  cluster_arrive();
  cluster_wait();
  if (w == 0) {
    // max|O_old|^2 over the cluster (FP64 maximum of the CTAs' FP64 patch
    // maxima), then the update strengths alpha / max|P|^2 and
    // beta / max|O_old|^2 (FP64 maxima, FP32 divisions), read by every
    // thread after the next barrier
    double omc = lane < S_CL ? oslot[lane] : 0.0;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) omc = fmax(omc, __shfl_xor_sync(0xffffffffu, omc, o));
    if (lane == 0) {
      const double om_used = a.omax2_global ? *a.omax2_global : omc;
      float *st = reinterpret_cast<float *>(smem + OFF_CAND);  // the candidates are consumed
      const float pmf = static_cast<float>(pm), omf = static_cast<float>(om_used);
      st[0] = pm > 0.0 ? a.alpha / pmf : 0.f;
      st[1] = om_used > 0.0 ? a.beta / omf : 0.f;
      st[2] = pm > 0.0 ? 1.0f / pmf : 0.f;
    }
  }

  // ---------------------------------------------------------------- phase 2
  // row stage A: thread (yl = lane, j = w), x = w + 16 r
#pragma unroll
  for (int r = 0; r < 32; ++r) EL(r) = slab[lane * RP + w + 16 * r];
  dft32<false>(lo, hi);
#pragma unroll
  for (int k1 = 1; k1 < 32; ++k1) EL(k1) = cmul(EL(k1), tw512<false>(w * k1));
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) slab[lane * RP + w + 16 * k1] = EL(k1);
  bool ok = mbar_wait_bounded(bar, 0, wait_ns);
  if (!ok) atomicOr(a.err_flag, FLAG_TMA_TIMEOUT);
  ok = __all_sync(0xffffffffu, ok);  // warp-uniform: phase 3 reads TMEM warp-collectively
  float isum_s = 0.f, isum_c = 0.f;  // sum I of this thread's converted values (raw path)
  if (!a.amp) {
    // raw rows -> sqrt(max(I - dark, 0)) in the amplitude layout, in place:
    // every raw value is read before the barrier, every float written after
    float iv[32];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int ci = tid + S_NT * u, yl = ci & 31, wm = ci >> 5;
      const int kx0 = 2 * (wm >> 3) + ((wm & 7) >> 2) + 128 * (wm & 3);
      const IT *row = reinterpret_cast<const IT *>(raw + yl * RawRows<IT>::PITCH);
#pragma unroll
      for (int i = 0; i < 4; ++i) iv[4 * u + i] = ival(row[kx0 + 32 * i]);
      if (a.dark) {
        const float *drow = a.dark + freq_of_pos(32 * c + yl) * S_N;
#pragma unroll
        for (int i = 0; i < 4; ++i) iv[4 * u + i] -= __ldg(drow + kx0 + 32 * i);
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 8; ++u) {
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
  // row stage B, modulus replacement, row stage B': thread (yl = lane),
  // k1 = 2 w (lo) and 2 w + 1 (hi)
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    lo[j] = slab[lane * RP + 32 * w + j];
    hi[j] = slab[lane * RP + 32 * w + 16 + j];
  }
  dft16<false>(lo);
  dft16<false>(hi);
  float e = 0.f;
  {
    // chunk (w * 8 + m) * 32 + yl holds the amplitudes of k1 = 2 w + (m >> 2),
    // k2 = 4 (m & 3) + i: element 4 m + i of (lo, hi)
    const float4 *a4 = reinterpret_cast<const float4 *>(ampt) + w * 8 * 32 + lane;
    constexpr float invK = 1.0f / (float(S_N) * float(S_N));
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const float4 s4 = a4[32 * m];
      const float sq[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float2 &z = EL(4 * m + i);
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
  dft16<true>(lo);
  dft16<true>(hi);
#pragma unroll
  for (int j = 1; j < 16; ++j) {
    lo[j] = cmul(lo[j], tw512<true>(j * 2 * w));
    hi[j] = cmul(hi[j], tw512<true>(j * (2 * w + 1)));
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    slab[lane * RP + 32 * w + j] = lo[j];
    slab[lane * RP + 32 * w + 16 + j] = hi[j];
  }
  {
    // error terms: FP32 over a thread's 32 elements, then an error-free
    // (two-sum) FP32 tree over the warp; FP64 only across warps, in one warp
    float eh = e, el = 0.f, sh = isum_s, sl = isum_c;
    warp_two_sum(eh, el);
    warp_two_sum(sh, sl);
    if (lane == 0) red[w] = make_float4(eh, el, sh, sl);
  }
  __syncthreads();
  // row stage A': thread (yl = lane, j = w)
  {
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) EL(k1) = slab[lane * RP + 16 * k1 + w];
    cluster_arrive();
    dft32<true>(lo, hi);
    cluster_wait();
    // x = w + 16 r goes to CTA r / 2, column w + 16 (r & 1), row position
    // 32 q + lane of its column-major tile: each warp store is one run of
    // 32 consecutive elements
    const uint32_t me = smem_u32(slab) + 8u * static_cast<uint32_t>(w * CT + 32 * c + lane);
#pragma unroll
    for (int r = 0; r < 32; ++r)
      st_cluster(map_rank(me + 8u * static_cast<uint32_t>(16 * (r & 1) * CT), static_cast<uint32_t>(r >> 1)),
                 EL(r));
  }
  cluster_arrive();
  cluster_wait();
  if (w == 0) {
    double es = 0.0, ss = 0.0;
    if (lane < S_NW) {
      const float4 t = red[lane];
      es = two_sum_value(t.x, t.y);
      ss = two_sum_value(t.z, t.w);
    }
    es = warp_sum_all(es);
    ss = warp_sum_all(ss);
    if (lane == 0) {
      a.err_part[static_cast<size_t>(f) * a.err_stride + c] = es;
      a.isum_part[static_cast<size_t>(f) * a.err_stride + c] =
          a.amp ? (c == 0 ? a.amp_isum[f] : 0.0) : ss;
    }
  }

  // ---------------------------------------------------------------- phase 3
  // column stage B': thread (b = lane), k1 = 2 w (lo) and 2 w + 1 (hi), tile
  // [column][row position]
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) {
    lo[k2] = slab[lane * CT + 32 * w + k2];
    hi[k2] = slab[lane * CT + 32 * w + 16 + k2];
  }
  dft16<true>(lo);
  dft16<true>(hi);
#pragma unroll
  for (int j = 1; j < 16; ++j) {
    lo[j] = cmul(lo[j], tw512<true>(j * 2 * w));
    hi[j] = cmul(hi[j], tw512<true>(j * (2 * w + 1)));
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    slab[lane * CT + 32 * w + j] = lo[j];
    slab[lane * CT + 32 * w + 16 + j] = hi[j];
  }
  __syncthreads();
  // column stage A': thread (b = lane, j = w) -> psi' at y = w + 16 r
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) EL(k1) = slab[lane * CT + 16 * k1 + w];
  dft32<true>(lo, hi);

  const float *st = reinterpret_cast<const float *>(smem + OFF_CAND);  // written after C2
  const float ao = st[0], bp = st[1];
  float2 *part = a.probe_part + static_cast<size_t>(member) * S_N * S_N + w * S_N + 32 * c + lane;
  if (ok) {
    if constexpr (!MB) {
      // the per-element scalings as paired-FP32 operations (each lane rounds
      // as the scalar fmaf / multiply would)
      const float2 ao2 = make_float2(ao, ao), bp2 = make_float2(bp, bp);
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        float ko[8], kp[8];  // four elements at a time keep the registers below the limit
        tmem_ld8(tm + 8 * h, ko);
        tmem_ld8(tm + 64 + 8 * h, kp);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = 4 * h + i;
          const float2 o = make_float2(ko[2 * i], ko[2 * i + 1]);
          const float2 p = make_float2(kp[2 * i], kp[2 * i + 1]);
          const float2 d = psub(EL(r), cmul(p, o));
          const float2 uo = cmulc(p, d);  // conj(P) Delta
          const float2 up = cmulc(o, d);  // conj(O_old) Delta
          st_l2hint(Ob + static_cast<size_t>(16 * r) * orow, __ffma2_rn(ao2, uo, o), opol);
          part[16 * r * S_N] = __fmul2_rn(up, bp2);
        }
      }
    } else {
      // mini-batch: patches of a batch may overlap; the object moves once per
      // batch by the count-normalised sum, applied by a separate kernel
      const float inv_pm = st[2];
      const size_t obase = static_cast<size_t>(py + w) * orow + px + 32 * c + lane;
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        float ko[8], kp[8];
        tmem_ld8(tm + 8 * h, ko);
        tmem_ld8(tm + 64 + 8 * h, kp);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = 4 * h + i;
          const float2 o = make_float2(ko[2 * i], ko[2 * i + 1]);
          const float2 p = make_float2(kp[2 * i], kp[2 * i + 1]);
          const float2 d = csub(EL(r), cmul(p, o));
          const float2 uo = cscale(cmulc(p, d), inv_pm);
          const size_t oi = obase + static_cast<size_t>(16 * r) * orow;
          atomicAdd(a.accO + oi, uo);  // one paired (8-byte) atomic
          atomicAdd(a.cnt + oi, 1);
          part[16 * r * S_N] = cscale(cmulc(o, d), bp);
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

#undef EL

// Measured amplitudes of frames [f0, f0 + n) in the layout of the step
// kernel's amplitude tiles: CTA q's tile (32 row positions p = 32 q + yl,
// frequency ky = (p >> 4) + 32 (p & 15)) holds, as float4 chunk
// (wq * 8 + m) * 32 + yl, the values at kx = k1 + 32 (4 (m & 3) + i),
// k1 = 2 wq + (m >> 2), i = 0..3.  amp = sqrt(max(I - dark, 0)); isum = sum
// of max(I - dark, 0), two-sum in FP32 per thread and a fixed-order FP64 sum
// over the block.  One block per frame walks the 16 tiles: each thread loads
// its chunks of the tile's 32 frequency rows as 16-byte vectors (TileLane),
// the next tile's loads are in flight while the current tile is written out
// chunk by chunk (coalesced).
constexpr int AI_NT = 512, AI_PITCH = S_N + 1;  // odd pitch: conflict-free chunk reads
constexpr size_t AI_SMEM = sizeof(float) * 32 * AI_PITCH + sizeof(double) * AI_NT;
template <typename IT>
__global__ void __launch_bounds__(AI_NT) amp_ingest512_kernel(const IT *__restrict__ frames,
                                                              const float *__restrict__ dark,
                                                              float *__restrict__ amp,
                                                              double *__restrict__ isum, int f0) {
  extern __shared__ __align__(16) unsigned char ai_smem[];
  float *rows = reinterpret_cast<float *>(ai_smem);
  double *sh = reinterpret_cast<double *>(ai_smem + sizeof(float) * 32 * AI_PITCH);
  const size_t fb = static_cast<size_t>(f0 + blockIdx.x) * S_N * S_N;
  const IT *fr = frames + fb;
  float4 *out = reinterpret_cast<float4 *>(amp + fb);
  const int t = threadIdx.x;
  float s = 0.f, cc = 0.f;
  TileLane<S_N, AI_NT, IT> tl;
  tl.load(fr, freq_of_pos(tl.yl));
  for (int q = 0; q < S_CL; ++q) {
    tl.store(rows, dark, freq_of_pos(32 * q + tl.yl), s, cc);
    __syncthreads();
    if (q + 1 < S_CL) tl.load(fr, freq_of_pos(32 * (q + 1) + tl.yl));
#pragma unroll
    for (int u = 0; u < 4096 / AI_NT; ++u) {
      const int cj = t + AI_NT * u, yl = cj & 31, wm = cj >> 5;
      const int kx0 = 2 * (wm >> 3) + ((wm & 7) >> 2) + 128 * (wm & 3);
      const float *r = rows + yl * AI_PITCH + kx0;
      out[q * 4096 + cj] = make_float4(r[0], r[32], r[64], r[96]);
    }
    __syncthreads();
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
cudaError_t launch_t(const GroupArgs &a, cudaStream_t st) {
  auto kern = epie_fused512_kernel<IT, MB>;
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_tw_ready[dev]) {
    // twiddles exp(-2 pi i m / 512), evaluated in double precision
    float2 tw[S_N];
    for (int m = 0; m < S_N; ++m) {
      const double ang = -2.0 * 3.14159265358979323846 * m / S_N;
      tw[m] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
    }
    cudaError_t e = cudaMemcpyToSymbol(c_tw512, tw, sizeof tw);
    if (e != cudaSuccess) return e;
    g_tw_ready[dev] = true;
  }
  if (!configured[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(SMEM512));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    // A TMEM allocation blocks until columns are free, and the CTAs of a
    // cluster wait for each other, so every CTA that can be resident on an
    // SM must find its 512 columns at once: exactly one resident CTA.
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, S_NT, SMEM512);
    if (e != cudaSuccess) return e;
    if (occ != 1) return cudaErrorInvalidConfiguration;
    configured[dev] = true;
  }
  if (a.n_members <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(a.n_members * S_CL), 1, 1);
  cfg.blockDim = dim3(S_NT, 1, 1);
  cfg.dynamicSmemBytes = SMEM512;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = S_CL;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <typename IT>
cudaError_t amp_ingest_t(const IT *frames, const float *dark, float *amp, double *isum, int f0, int n,
                         cudaStream_t st) {
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!configured[dev]) {
    cudaError_t e = cudaFuncSetAttribute(amp_ingest512_kernel<IT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(AI_SMEM));
    if (e != cudaSuccess) return e;
    configured[dev] = true;
  }
  amp_ingest512_kernel<IT><<<n, AI_NT, AI_SMEM, st>>>(frames, dark, amp, isum, f0);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fused_512(int itype, const GroupArgs &a, cudaStream_t st) {
  // the mini-batch update (object-update accumulator) is its own instantiation
  const bool mb = a.accO != nullptr;
  if (itype == 0) return mb ? launch_t<uint16_t, true>(a, st) : launch_t<uint16_t, false>(a, st);
  if (itype == 1) return mb ? launch_t<__half, true>(a, st) : launch_t<__half, false>(a, st);
  return mb ? launch_t<float, true>(a, st) : launch_t<float, false>(a, st);
}

size_t fused_smem_512(int /*itype*/) { return SMEM512; }

cudaError_t launch_amp_ingest_512(const void *frames, int itype, const float *dark, float *amp,
                                  double *isum, int f0, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (itype == 0) return amp_ingest_t(static_cast<const uint16_t *>(frames), dark, amp, isum, f0, n, st);
  if (itype == 1) return amp_ingest_t(static_cast<const __half *>(frames), dark, amp, isum, f0, n, st);
  return amp_ingest_t(static_cast<const float *>(frames), dark, amp, isum, f0, n, st);
}

}  // namespace epie
