// epie_fused_256.cu -- the fused ePIE position-update kernel for 256 x 256
// frames, and the measured-amplitude layout it reads.
//
// One thread-block cluster of 8 CTAs x 512 threads owns one scan position of
// a group (the ePIE step of Maiden & Rodenburg 2009, as the paper's engine
// runs it, Sec. "ePIE Implementation"; alpha = beta = 1 in the paper).  The
// 2-D transform runs as radix-16 stages over 256 = 16 x 16 along each axis,
// written so that every stage reads and writes the same set of elements of
// each thread (no barrier between the loads and the stores of a stage):
//
//   forward (decimation in frequency), for n = j + 16 r, k = k1 + 16 k2:
//     stage A  thread j: Y[k1] = sum_r x[j + 16 r] W16^(r k1), times
//              W256^(j k1), stored at j + 16 k1;
//     stage B  thread k1: X[k1 + 16 k2] = sum_j Y[j + 16 k1] W16^(j k2),
//              stored at 16 k1 + k2 (the spectrum in digit-reversed order);
//   inverse (decimation in time) from that order back to natural order:
//     stage B' thread k1: Z[j] = sum_k2 X'[16 k1 + k2] W16^(-j k2), times
//              W256^(-j k1), stored at 16 k1 + j;
//     stage A' thread j: x'[j + 16 r] = sum_k1 Z[16 k1 + j] W16^(-r k1).
//
//   phase 1  CTA c, columns [32c, 32c + 32): each thread loads the object
//            patch and probe of its 16 elements (x = 32c + lane, y = w + 16r,
//            w = warp) straight into registers, parks them in tensor memory,
//            forms psi = P . O_j and runs column stage A; then column stage B
//            and a push of the finished column spectra into the peer CTA
//            that owns their row block (st.shared::cluster, between split
//            cluster barriers: the peers' tiles are free once every CTA has
//            loaded its stage-B inputs);
//   phase 2  CTA q, row positions [32q, 32q + 32): row stage A, then row
//            stage B, the modulus replacement with sqrt(I) (the measured
//            amplitude tile, in the order of the digit-reversed spectrum,
//            arrives by one bulk copy issued at kernel start) and row stage
//            B' in registers, then row stage A' and a push of the rows back
//            to the column owners;
//   phase 3  column stages B' and A' give psi' for exactly the 16 elements
//            each thread loaded in phase 1, so Delta = psi' - psi, the
//            object update with conj(P)/max|P|^2 (patches of a group are
//            disjoint, so the writes never race) and the probe-update
//            partial beta conj(O_old)/max|O_old|^2 Delta are formed in
//            registers, with O_old and P read back from tensor memory.
//
// Shared memory holds the CTA's tile (phase 1 [row position][33], phase 2
// [row][257], phase 3 [column][257] complex: odd pitches keep every stage
// free of bank conflicts, and both pushes write runs of 32 consecutive
// elements per warp, the fast pattern for distributed shared memory),
// the amplitude tile and a few reduction slots: 2 CTAs per SM.  Twiddles
// W256^m are in constant memory; every twiddle index is warp-uniform.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "epie_cluster.cuh"
#include "epie_fft.cuh"
#include "epie_ingest.cuh"
#include "epie_internal.h"

namespace epie {

// Phase clocks for profiling builds only (-DEPIE_PHASE_CLOCKS): thread 0 of
// each CTA records clock64() at the phase boundaries; normal builds compile
// the markers to nothing.
#ifdef EPIE_PHASE_CLOCKS
// slots 0..11: clock64() at the phase markers; 12: SM id; 13, 14: %globaltimer
// at the first and the last marker (comparable across SMs)
static __device__ long long g_phase_clocks[4096][16];
#define EPIE_PHASE(k)                                                                        \
  do {                                                                                       \
    if (threadIdx.x == 0 && blockIdx.x < 4096) {                                             \
      g_phase_clocks[blockIdx.x][k] = clock64();                                             \
      if ((k) == 0 || (k) == 11) {                                                           \
        uint32_t smid_;                                                                      \
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid_));                                   \
        g_phase_clocks[blockIdx.x][12] = smid_;                                              \
        g_phase_clocks[blockIdx.x][(k) == 0 ? 13 : 14] = static_cast<long long>(global_ns()); \
      }                                                                                      \
    }                                                                                        \
  } while (0)
#else
#define EPIE_PHASE(k) \
  do {                \
  } while (0)
#endif

namespace {

constexpr int S_N = 256, S_CL = 8, S_NT = 512, S_NW = 16;
// clusters (frames) one wave of this kernel holds on a GB300 (2 CTAs per SM;
// measured: the first wave of a 65-member group started 35 clusters)
constexpr int S_WAVE = 35;
static_assert(EPIE_CTAS_256 == S_CL, "the 256^2 kernel runs 8-CTA clusters");
constexpr int CP = 33;                       // column-tile pitch (complex)
constexpr int RP = 257;                      // row-tile pitch (complex)
constexpr int CT = 257;                      // phase-3 tile: [column][row position]
constexpr int SLAB = S_N * CP;               // >= 32 * RP
constexpr size_t OFF_AMP = sizeof(float2) * SLAB;
constexpr uint32_t AMP_BYTES = 32 * S_N * sizeof(float);  // one CTA's amplitude tile
constexpr size_t STAGE_BYTES = 32 * (S_N * 4 + 16);       // raw rows of any type, padded
constexpr size_t OFF_RED = OFF_AMP + STAGE_BYTES;         // 2 doubles per warp (4 floats)
constexpr size_t OFF_OMAX = OFF_RED + sizeof(double) * 2 * S_NW;  // 8 cluster slots
constexpr size_t OFF_CAND = OFF_OMAX + sizeof(double) * S_CL;     // float4 per warp
constexpr size_t OFF_BAR = OFF_CAND + 16 * S_NW;
constexpr size_t SMEM256 = OFF_BAR + 16;  // mbarrier, then the TMEM address slot
constexpr int TM_COLS = 256;              // 64 columns per thread, 4 warps per lane quadrant
static_assert(32 * RP <= SLAB && 32 * CT <= SLAB, "row and phase-3 tiles fit the slab");
static_assert(OFF_AMP % 16 == 0 && OFF_RED % 16 == 0 && OFF_CAND % 16 == 0 && OFF_BAR % 8 == 0,
              "alignment of the shared-memory regions");

// raw intensity rows (allocation-free entry point): 32 rows of 256 values,
// row pitch a multiple of 16 bytes (bulk-copy destinations)
template <typename IT>
struct RawRows {
  static constexpr int PITCH = S_N * static_cast<int>(sizeof(IT)) + 16;
  static_assert(32 * PITCH <= static_cast<int>(STAGE_BYTES), "raw rows fit the staging area");
};

__constant__ float2 c_tw256[S_N];  // exp(-2 pi i m / 256)

// row position p of the digit-reversed spectrum holds frequency
// (p >> 4) + 16 (p & 15)
__device__ __forceinline__ int freq_of_pos(int p) { return (p >> 4) + 16 * (p & 15); }

template <bool INV>
__device__ __forceinline__ float2 tw256(int m) {
  float2 w = c_tw256[m];
  if (INV) w.y = -w.y;
  return w;
}


template <typename IT, bool MB>
__global__ void __launch_bounds__(S_NT, 2) epie_fused256_kernel(GroupArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  float2 *slab = reinterpret_cast<float2 *>(smem);
  float *ampt = reinterpret_cast<float *>(smem + OFF_AMP);
  double *red = reinterpret_cast<double *>(smem + OFF_RED);
  double *oslot = reinterpret_cast<double *>(smem + OFF_OMAX);
  float4 *cand = reinterpret_cast<float4 *>(smem + OFF_CAND);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + OFF_BAR);
  uint32_t *tm_slot = reinterpret_cast<uint32_t *>(smem + OFF_BAR + 8);

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  EPIE_PHASE(0);
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
  // this thread's tensor-memory columns: [0, 32) object patch, [32, 64) probe
  const uint32_t tm = *tm_slot + (static_cast<uint32_t>(32 * (w & 3)) << 16) +
                      static_cast<uint32_t>((w >> 2) * 64);
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
  float2 v[16];
  float om = -1.f;
  float2 omv = make_float2(0.f, 0.f);
  auto load_patch = [&]() {
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = ld_l2hint(Ob + static_cast<size_t>(16 * r) * orow, opol);
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
  };
  // A group larger than one wave of clusters runs a second wave: warm L2 with
  // the object rows of the frame that will take this cluster's place there
  // (a hint only; a prefetch of lines still being written is harmless).
  if (member + S_WAVE < n_members && tid < S_N) {
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
  load_patch();
  if (a.o_early) grid_dependency_wait();
  grid_dependents_launch();
  if (blockIdx.x == 0 && tid == 0 && a.pmax2_clear) *a.pmax2_clear = 0ull;
  // max|P|^2 of the group (written by the preceding reduction), fetched
  // early: the update strengths are formed after the first transpose
  double pm = 0.0;
  if (tid == 0) pm = __longlong_as_double(static_cast<long long>(*a.pmax2));
  // the probe: with the object values parked, v takes all 16 probe values in
  // one round trip; the exit wave multiplies the parked object values back in
  tmem_wait_st();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = __ldg(Pb + r * 16 * S_N);
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
  EPIE_PHASE(1);
  // column stage A
  dft<16, false>(v);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], tw256<false>(w * k1));
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) slab[(w + 16 * k1) * CP + lane] = v[k1];
  // max |O_old|^2 over the patch: FP32 comparisons pick the element (lanes,
  // warps, then CTAs); its square is formed in FP64
  omv = warp_argmax_f(om, omv);
  if (lane == 0) cand[w] = make_float4(omv.x, omv.y, omv.x * omv.x + omv.y * omv.y, 0.f);
  tmem_wait_st();
  __syncthreads();
  EPIE_PHASE(2);
  // column stage B: thread (b = lane, k1 = w)
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = slab[(16 * w + j) * CP + lane];
  cluster_arrive();  // this CTA's tile is free once every thread has its inputs
  dft<16, false>(v);
  double om_cta = 0.0;
  if (w == 0) {
    float4 cd = lane < S_NW ? cand[lane] : make_float4(0.f, 0.f, -1.f, 0.f);
    const float2 cv = warp_argmax_f(cd.z, make_float2(cd.x, cd.y));
    om_cta = static_cast<double>(cv.x) * cv.x + static_cast<double>(cv.y) * cv.y;
  }
  cluster_wait();
  EPIE_PHASE(3);
  {
    // spectrum rows p = 16 k1 + k2 go to CTA k1 / 2, local row 16 (k1 & 1) + k2
    const uint32_t dst = map_rank(smem_u32(slab), static_cast<uint32_t>(w >> 1));
    const uint32_t base = dst + 8u * static_cast<uint32_t>((16 * (w & 1)) * RP + 32 * c + lane);
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) st_cluster(base + 8u * static_cast<uint32_t>(k2 * RP), v[k2]);
    if (w == 0 && lane < S_CL)
      st_cluster(map_rank(smem_u32(oslot + c), static_cast<uint32_t>(lane)), om_cta);
  }
  cluster_arrive();
  cluster_wait();
  EPIE_PHASE(4);
  if (w == 0) {
    // max|O_old|^2 over the cluster (FP64 maximum of the CTAs' FP64 patch
    // maxima), then the update strengths alpha / max|P|^2 and
    // beta / max|O_old|^2; the maxima stay FP64, the divisions are FP32 (the
    // FP64 pipe is narrow); read by every thread after the next barrier
    double om = lane < S_CL ? oslot[lane] : 0.0;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) om = fmax(om, __shfl_xor_sync(0xffffffffu, om, o));
    if (lane == 0) {
      const double om_used = a.omax2_global ? *a.omax2_global : om;
      float *st = reinterpret_cast<float *>(smem + OFF_CAND);  // the candidates are consumed
      const float pmf = static_cast<float>(pm), omf = static_cast<float>(om_used);
      st[0] = pm > 0.0 ? a.alpha / pmf : 0.f;
      st[1] = om_used > 0.0 ? a.beta / omf : 0.f;
      st[2] = pm > 0.0 ? 1.0f / pmf : 0.f;
    }
  }

  // ---------------------------------------------------------------- phase 2
  // row stage A: thread (yl = lane, j = w)
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = slab[lane * RP + w + 16 * r];
  dft<16, false>(v);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], tw256<false>(w * k1));
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) slab[lane * RP + w + 16 * k1] = v[k1];
  bool ok = mbar_wait_bounded(bar, 0, wait_ns);
  if (!ok) atomicOr(a.err_flag, FLAG_TMA_TIMEOUT);
  ok = __all_sync(0xffffffffu, ok);  // warp-uniform: phase 3 reads TMEM warp-collectively
  float isum_s = 0.f, isum_c = 0.f;  // sum I of this thread's converted values (raw path)
  if (!a.amp) {
    // raw rows -> sqrt(max(I - dark, 0)) in the amplitude layout, in place:
    // every raw value is read before the barrier, every float written after
    float iv[16];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int ci = tid + S_NT * u, yl = ci & 31, k1m = ci >> 5;
      const int k1 = k1m >> 2, m = k1m & 3;
      const IT *row = reinterpret_cast<const IT *>(raw + yl * RawRows<IT>::PITCH);
#pragma unroll
      for (int i = 0; i < 4; ++i) iv[4 * u + i] = ival(row[k1 + 16 * (4 * m + i)]);
      if (a.dark) {
        const float *drow = a.dark + freq_of_pos(32 * c + yl) * S_N;
#pragma unroll
        for (int i = 0; i < 4; ++i) iv[4 * u + i] -= __ldg(drow + k1 + 16 * (4 * m + i));
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
  EPIE_PHASE(5);
  // row stage B, modulus replacement, row stage B': thread (yl = lane, k1 = w)
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = slab[lane * RP + 16 * w + j];
  dft<16, false>(v);
  float e = 0.f;
  {
    const float4 *a4 = reinterpret_cast<const float4 *>(ampt) + w * 4 * 32 + lane;
    constexpr float invK = 1.0f / (float(S_N) * float(S_N));
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const float4 s4 = a4[32 * m];
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
  dft<16, true>(v);
#pragma unroll
  for (int j = 1; j < 16; ++j) v[j] = cmul(v[j], tw256<true>(w * j));
#pragma unroll
  for (int j = 0; j < 16; ++j) slab[lane * RP + 16 * w + j] = v[j];
  {
    // error terms: FP32 over a thread's 16 elements, then an error-free
    // (two-sum) FP32 tree over the warp; FP64 only across warps, in one warp
    float eh = e, el = 0.f, sh = isum_s, sl = isum_c;
    warp_two_sum(eh, el);
    warp_two_sum(sh, sl);
    if (lane == 0) reinterpret_cast<float4 *>(red)[w] = make_float4(eh, el, sh, sl);
  }
  __syncthreads();
  EPIE_PHASE(6);
  // row stage A': thread (yl = lane, j = w)
  {
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) v[k1] = slab[lane * RP + w + 16 * k1];
    cluster_arrive();
    dft<16, true>(v);
    cluster_wait();
    EPIE_PHASE(7);
    // x = w + 16 r goes to CTA r / 2, column w + 16 (r & 1), row position
    // 32 q + lane of its column-major tile: each warp store is one run of
    // 32 consecutive elements
    const uint32_t me = smem_u32(slab) + 8u * static_cast<uint32_t>(w * CT + 32 * c + lane);
#pragma unroll
    for (int r = 0; r < 16; ++r)
      st_cluster(map_rank(me + 8u * static_cast<uint32_t>(16 * (r & 1) * CT), static_cast<uint32_t>(r >> 1)),
                 v[r]);
  }
  cluster_arrive();
  cluster_wait();
  EPIE_PHASE(8);
  if (w == 0) {
    double es = 0.0, ss = 0.0;
    if (lane < S_NW) {
      const float4 t = reinterpret_cast<const float4 *>(red)[lane];
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
  // column stage B': thread (b = lane, k1 = w), tile [column][row position]
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) v[k2] = slab[lane * CT + 16 * w + k2];
  dft<16, true>(v);
#pragma unroll
  for (int j = 1; j < 16; ++j) v[j] = cmul(v[j], tw256<true>(w * j));
#pragma unroll
  for (int j = 0; j < 16; ++j) slab[lane * CT + 16 * w + j] = v[j];
  __syncthreads();
  EPIE_PHASE(9);
  // column stage A': thread (b = lane, j = w) -> psi' at y = w + 16 r
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) v[k1] = slab[lane * CT + w + 16 * k1];
  dft<16, true>(v);
  EPIE_PHASE(10);

  const float *st = reinterpret_cast<const float *>(smem + OFF_CAND);  // written after C2
  const float ao = st[0], bp = st[1];
  float2 *part = a.probe_part + static_cast<size_t>(member) * S_N * S_N + w * S_N + 32 * c + lane;
  if (ok) {
    if constexpr (!MB) {
      // the per-element scalings as paired-FP32 operations (each lane rounds
      // as the scalar fmaf / multiply would)
      const float2 ao2 = make_float2(ao, ao), bp2 = make_float2(bp, bp);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float ko[8], kp[8];  // four elements at a time keep the registers below the limit
        tmem_ld8(tm + 8 * h, ko);
        tmem_ld8(tm + 32 + 8 * h, kp);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = 4 * h + i;
          const float2 o = make_float2(ko[2 * i], ko[2 * i + 1]);
          const float2 p = make_float2(kp[2 * i], kp[2 * i + 1]);
          const float2 d = psub(v[r], cmul(p, o));
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
      for (int h = 0; h < 4; ++h) {
        float ko[8], kp[8];
        tmem_ld8(tm + 8 * h, ko);
        tmem_ld8(tm + 32 + 8 * h, kp);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = 4 * h + i;
          const float2 o = make_float2(ko[2 * i], ko[2 * i + 1]);
          const float2 p = make_float2(kp[2 * i], kp[2 * i + 1]);
          const float2 d = csub(v[r], cmul(p, o));
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
  EPIE_PHASE(11);
  if (w == 0) {
    tc_fence_after();
    tmem_dealloc(*tm_slot, TM_COLS);
  }
}

// Measured amplitudes of frames [f0, f0 + n) in the layout of the step
// kernel's amplitude tiles: CTA q's tile (32 row positions p = 32 q + yl,
// frequency ky = (p >> 4) + 16 (p & 15)) holds, as float4 chunk
// (k1 * 4 + m) * 32 + yl, the values at kx = k1 + 16 (4 m + i), i = 0..3.
// amp = sqrt(max(I - dark, 0)); isum = sum of max(I - dark, 0), two-sum in
// FP32 per thread and a fixed-order FP64 sum over the block.  One block per
// frame walks the 8 tiles: each thread loads its chunks of the tile's 32
// frequency rows as 16-byte vectors (TileLane), the next tile's loads are in
// flight while the current tile is written out chunk by chunk (coalesced).
constexpr int AI_NT = 256, AI_PITCH = S_N + 1;  // odd pitch: conflict-free chunk reads
template <typename IT>
__global__ void __launch_bounds__(AI_NT) amp_ingest256_kernel(const IT *__restrict__ frames,
                                                              const float *__restrict__ dark,
                                                              float *__restrict__ amp,
                                                              double *__restrict__ isum, int f0) {
  __shared__ float rows[32 * AI_PITCH];
  __shared__ double sh[AI_NT];
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
    for (int u = 0; u < 2048 / AI_NT; ++u) {
      const int cj = t + AI_NT * u, yl = cj & 31, k1m = cj >> 5;
      const int k1 = k1m >> 2, m = k1m & 3;
      const float *r = rows + yl * AI_PITCH + k1 + 64 * m;
      out[q * 2048 + cj] = make_float4(r[0], r[16], r[32], r[48]);
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
  auto kern = epie_fused256_kernel<IT, MB>;
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_tw_ready[dev]) {
    // twiddles exp(-2 pi i m / 256), evaluated in double precision
    float2 tw[S_N];
    for (int m = 0; m < S_N; ++m) {
      const double ang = -2.0 * 3.14159265358979323846 * m / S_N;
      tw[m] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
    }
    cudaError_t e = cudaMemcpyToSymbol(c_tw256, tw, sizeof tw);
    if (e != cudaSuccess) return e;
    g_tw_ready[dev] = true;
  }
  if (!configured[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(SMEM256));
    if (e != cudaSuccess) return e;
    // prefer the whole unified L1 / shared-memory array as shared memory
    // (2 resident CTAs of this size)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    // A TMEM allocation blocks until columns are free, and the CTAs of a
    // cluster wait for each other, so every CTA that can be resident on an
    // SM must find its 256 columns at once: at most 2 resident CTAs.
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, S_NT, SMEM256);
    if (e != cudaSuccess) return e;
    if (occ < 1 || occ * TM_COLS > 512) return cudaErrorInvalidConfiguration;
    configured[dev] = true;
  }
  if (a.n_members <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(a.n_members * S_CL), 1, 1);
  cfg.blockDim = dim3(S_NT, 1, 1);
  cfg.dynamicSmemBytes = SMEM256;
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

}  // namespace

cudaError_t launch_fused_256(int itype, const GroupArgs &a, cudaStream_t st) {
  // the mini-batch update (object-update accumulator) is its own instantiation
  const bool mb = a.accO != nullptr;
  if (itype == 0) return mb ? launch_t<uint16_t, true>(a, st) : launch_t<uint16_t, false>(a, st);
  if (itype == 1) return mb ? launch_t<__half, true>(a, st) : launch_t<__half, false>(a, st);
  return mb ? launch_t<float, true>(a, st) : launch_t<float, false>(a, st);
}

size_t fused_smem_256(int /*itype*/) { return SMEM256; }

cudaError_t launch_amp_ingest_256(const void *frames, int itype, const float *dark, float *amp,
                                  double *isum, int f0, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (itype == 0)
    amp_ingest256_kernel<<<n, AI_NT, 0, st>>>(static_cast<const uint16_t *>(frames), dark, amp,
                                             isum, f0);
  else if (itype == 1)
    amp_ingest256_kernel<<<n, AI_NT, 0, st>>>(static_cast<const __half *>(frames), dark, amp,
                                             isum, f0);
  else
    amp_ingest256_kernel<<<n, AI_NT, 0, st>>>(static_cast<const float *>(frames), dark, amp,
                                             isum, f0);
  return cudaGetLastError();
}

}  // namespace epie

#ifdef EPIE_PHASE_CLOCKS
// profiling builds: copy the per-CTA phase clocks of the last launch to the host
extern "C" __attribute__((visibility("default"))) int epie_read_phase_clocks(long long *host,
                                                                            int n_ctas) {
  return static_cast<int>(
      cudaMemcpyFromSymbol(host, epie::g_phase_clocks, sizeof(long long) * 16 * n_ctas));
}
#endif
