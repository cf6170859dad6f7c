// epie_fused.cuh -- the fused ePIE position-update kernel.
//
// One thread-block cluster of CL CTAs owns one scan position of a group
// (ePIE step, Maiden & Rodenburg 2009, as run by the paper's engine, Sec.
// "ePIE Implementation"; alpha = beta = 1 in the paper):
//
//   phase 1  CTA c forms the exit wave psi = P . O_j on the column block
//            [c N/CL, (c+1) N/CL) and transforms every column (FFT along y);
//   swap     all-to-all transpose through distributed shared memory: CTA c
//            now holds the row block [c N/CL, (c+1) N/CL) of the spectrum;
//   phase 2  FFT along x, modulus replacement with sqrt(I) (the frame's
//            measured-amplitude tile, derived at append, arrives by a bulk
//            TMA copy issued at kernel start; without derived amplitudes the
//            raw intensity tile is copied and converted here, dark field
//            subtracted), error terms summed, inverse FFT along x;
//   swap     transpose back to column blocks;
//   phase 3  inverse FFT along y -> psi', Delta = psi' - psi, object patch
//            update with conj(P)/max|P|^2 (patches of a group are disjoint, so
//            the writes never race) and the probe-update partial
//            beta conj(O_old)/max|O_old|^2 Delta for the group reduction;
//            the object patch and probe values of phase 1 come back from
//            tensor memory, where each thread parked them.
//
// At N = 64 one CTA holds the whole frame (CL = 1) and the swaps are plain
// shared-memory re-indexing.  Shared memory holds one tile per CTA, the
// twiddle table, the amplitude (or intensity) tile and a few reduction
// slots.
#pragma once

#include <cooperative_groups.h>

#include "epie_fft.cuh"
#include "epie_internal.h"

namespace epie {

namespace cg = cooperative_groups;

// Phase clocks for profiling builds only (-DEPIE_PHASE_CLOCKS): thread 0 of
// each CTA records clock64() at the phase boundaries; normal builds compile
// the markers to nothing.
#ifdef EPIE_PHASE_CLOCKS
static __device__ long long g_phase_clocks[4096][16];
#define EPIE_PHASE(k)                                                        \
  do {                                                                       \
    if (threadIdx.x == 0 && blockIdx.x < 4096) g_phase_clocks[blockIdx.x][k] = clock64(); \
  } while (0)
#else
#define EPIE_PHASE(k) \
  do {                \
  } while (0)
#endif

template <int N, int CL, int NT, typename IT>
struct FusedCfg {
  static constexpr int WC = N / CL;        // columns per CTA in phases 1 and 3
  static constexpr int HR = N / CL;        // rows per CTA in phase 2
  static constexpr int PB = N + N / 16;    // padded row pitch of the row tile
  static constexpr int E = N * WC / NT;    // elements per thread, phases 1 and 3
  static constexpr int NW = NT / 32;
  static constexpr int SLAB =
      CL == 1 ? N * PB : (N * WC > HR * PB ? N * WC : HR * PB);  // float2 elements
  static constexpr size_t OFF_TW = sizeof(float2) * SLAB;
  static constexpr size_t OFF_I = OFF_TW + sizeof(float2) * N;  // float I_eff tile
  static constexpr uint32_t I_BYTES = HR * N * sizeof(IT);        // raw tile (bulk copy)
  static constexpr uint32_t IF_BYTES = HR * N * sizeof(float);
  static constexpr size_t OFF_IRAW = OFF_I + IF_BYTES - I_BYTES;  // raw tile at the top
  static constexpr size_t OFF_RED = (OFF_I + IF_BYTES + 15) / 16 * 16;
  static constexpr size_t OFF_BAR = OFF_RED + sizeof(double) * (2 * NW + 2);
  static constexpr size_t SMEM = OFF_BAR + 16;  // mbarrier, then the TMEM address slot
  // tensor memory: 64 columns per thread (32 for its object-patch values,
  // 32 for its probe values) in its warp's lane quadrant
  static constexpr int TM_COLS = (NW / 4) * 64;
  static_assert(E == 16, "16 complex values per thread fill 32 TMEM columns");
  static_assert(NW % 4 == 0 && (TM_COLS & (TM_COLS - 1)) == 0 && TM_COLS >= 32 &&
                    TM_COLS <= 512,
                "TMEM allocation is a power of two between 32 and 512 columns");
  static_assert(E * NT == N * WC, "tile must split evenly over threads");
  static_assert(I_BYTES % 16 == 0, "bulk copy size");
  static_assert(OFF_IRAW % 16 == 0, "bulk copy destination alignment");
  static_assert(OFF_I % 16 == 0 && IF_BYTES % 16 == 0, "amplitude tile bulk copy");
};

template <int N>
struct ModReplace {
  const float *sqtile;  // HR x N values sqrt(max(I - dark, 0)) of this CTA's rows
  float e;              // sum (|Psi| - sqrt I)^2 (FP32 per thread)
  __device__ __forceinline__ float2 operator()(int b, int kx, float2 v) {
    const float sq = sqtile[b * N + kx];
    const float a2 = v.x * v.x + v.y * v.y;
    constexpr float invK = 1.0f / (float(N) * float(N));
    float2 out;
    float amp;
    if (a2 > 0.f) {
      const float ia = rsqrtf(a2);
      amp = a2 * ia;
      const float r = sq * ia * invK;
      out = make_float2(v.x * r, v.y * r);
    } else {
      amp = 0.f;
      out = make_float2(sq * invK, 0.f);
    }
    const float d = amp - sq;
    e = fmaf(d, d, e);
    return out;
  }
};

// resident CTAs per SM the register budget is sized for
template <int CL, int NT>
constexpr int fused_min_blocks() {
#ifdef EPIE_FUSED_MIN_BLOCKS
  return EPIE_FUSED_MIN_BLOCKS;
#else
  return CL == 1 && NT <= 256 ? 2 : (1024 / NT > 1 ? 1024 / NT : 1);
#endif
}

template <int N, int CL, int NT, typename IT>
__global__ void __launch_bounds__(NT, fused_min_blocks<CL, NT>()) epie_fused_kernel(GroupArgs a) {
  using C = FusedCfg<N, CL, NT, IT>;
  constexpr int WC = C::WC, HR = C::HR, PB = C::PB, E = C::E, NW = C::NW;
  using ColA = ColAddr<CL == 1 ? PB : WC, CL == 1>;
  using RowB = RowAddr<PB>;

  extern __shared__ __align__(128) unsigned char smem[];
  float2 *slab = reinterpret_cast<float2 *>(smem);
  float2 *tw = reinterpret_cast<float2 *>(smem + C::OFF_TW);
  float *itile = reinterpret_cast<float *>(smem + C::OFF_I);
  IT *iraw = reinterpret_cast<IT *>(smem + C::OFF_IRAW);
  double *red = reinterpret_cast<double *>(smem + C::OFF_RED);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + C::OFF_BAR);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  EPIE_PHASE(0);
  const int member = blockIdx.x / CL;
  const int32_t *members = a.members;
  if (a.gstart) {
    // device group table: a whole cluster past the group's size exits here,
    // before any barrier or copy
    const int g0 = a.gstart[a.group];
    if (member >= a.gstart[a.group + 1] - g0) return;
    members += g0;
  }
  int crank = 0;
  if constexpr (CL > 1) crank = static_cast<int>(cg::this_cluster().block_rank());
  const int f = members[member];
  const int py = a.pos[2 * f], px = a.pos[2 * f + 1];
  const IT *frame = static_cast<const IT *>(a.frames) + static_cast<size_t>(f) * N * N;

  // The object patch and probe values a thread reads in phase 1 are kept in
  // tensor memory (unused otherwise by this kernel) until phase 3 needs them
  // again, instead of being re-read from L2 / HBM.  Warp 0 allocates.
  uint32_t *tm_slot = reinterpret_cast<uint32_t *>(smem + C::OFF_BAR + 8);
  if (warp == 0) tmem_alloc(tm_slot, C::TM_COLS);
  // intensity rows [crank*HR, +HR) of the frame: one bulk copy, waited on
  // just before the modulus replacement
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm_base = *tm_slot;
  // this thread's columns: [0, 32) object patch, [32, 64) probe
  const uint32_t tm = tm_base + (static_cast<uint32_t>(32 * (warp & 3)) << 16) +
                      static_cast<uint32_t>((warp >> 2) * 64);
  const uint64_t wait_ns = a.wait_ns ? a.wait_ns : 2000000000ull;
  // (failure injection: the launch's first CTA never issues its copy)
  if (tid == 0 && !(a.inject_skip_copy && blockIdx.x == 0)) {
    // the frame is read once per sweep: keep it from evicting the object.
    // With derived amplitudes the tile arrives ready for the modulus.
    if (a.amp) {
      mbar_arrive_expect_tx(bar, C::IF_BYTES);
      bulk_g2s_hint(itile, a.amp + static_cast<size_t>(f) * N * N + static_cast<size_t>(crank) * HR * N,
                    C::IF_BYTES, bar, l2_evict_first_policy());
    } else {
      mbar_arrive_expect_tx(bar, C::I_BYTES);
      bulk_g2s_hint(iraw, frame + static_cast<size_t>(crank) * HR * N, C::I_BYTES, bar,
                    l2_evict_first_policy());
    }
  }
  for (int m = tid; m < N; m += NT) tw[m] = a.twiddle[m];

  // ---------------------------------------------------------------- phase 1
  const size_t orow = static_cast<size_t>(a.W);
  float2 *Obase = a.O + static_cast<size_t>(py) * orow + px + crank * WC;
  const float2 *Pbase = a.P + crank * WC;
  float om = -1.f;
  float2 omv = make_float2(0.f, 0.f);
#ifndef EPIE_LOAD_BATCH
#define EPIE_LOAD_BATCH 8
#endif
  constexpr int EB = E >= EPIE_LOAD_BATCH ? EPIE_LOAD_BATCH : E;  // loads in flight together
#ifndef EPIE_NO_OBJECT_L2_HINT
  // the object is revisited by every later class: keep it in L2 ahead of the
  // streamed frames and the probe partials
  const uint64_t opol = l2_evict_last_policy();
#define EPIE_LD_O(p) ld_l2hint((p), opol)
#define EPIE_ST_O(p, v) st_l2hint((p), (v), opol)
#else
#define EPIE_LD_O(p) (*(p))
#define EPIE_ST_O(p, v) (*(p) = (v))
#endif
  // the object patch goes to the tile (and its maximum is found) before the
  // dependency wait when o_early says it is final, after it otherwise; the
  // probe, written by the preceding reduction, is applied after the wait
  auto load_patch = [&]() {
#pragma unroll
    for (int i0 = 0; i0 < E; i0 += EB) {
      float2 ov[EB];
#pragma unroll
      for (int i = 0; i < EB; ++i) {
        const int idx = tid + (i0 + i) * NT, y = idx / WC, xl = idx % WC;
        ov[i] = EPIE_LD_O(Obase + y * orow + xl);
      }
      float keep[2 * EB];
#pragma unroll
      for (int i = 0; i < EB; ++i) {
        const int idx = tid + (i0 + i) * NT, y = idx / WC, xl = idx % WC;
        const float q = ov[i].x * ov[i].x + ov[i].y * ov[i].y;
        if (q > om) { om = q; omv = ov[i]; }
        slab[ColA::at(xl, y)] = ov[i];
        keep[2 * i] = ov[i].x;
        keep[2 * i + 1] = ov[i].y;
      }
      tmem_st16(tm + 2 * i0, keep);
    }
  };
  if (a.o_early) load_patch();
  // everything above reads data written before the sweep (or, with o_early,
  // an object no kernel still running writes); the probe, max|P|^2 and the
  // partial buffers are written by the preceding kernels
  grid_dependency_wait();
  grid_dependents_launch();
  if (blockIdx.x == 0 && tid == 0 && a.pmax2_clear) *a.pmax2_clear = 0ull;
  if (!a.o_early) load_patch();
#pragma unroll
  for (int i0 = 0; i0 < E; i0 += EB) {
    float2 pv[EB];
#pragma unroll
    for (int i = 0; i < EB; ++i) {
      const int idx = tid + (i0 + i) * NT, y = idx / WC, xl = idx % WC;
      pv[i] = __ldg(Pbase + y * N + xl);
    }
    float keep[2 * EB];
#pragma unroll
    for (int i = 0; i < EB; ++i) {
      const int idx = tid + (i0 + i) * NT, y = idx / WC, xl = idx % WC;
      float2 &t = slab[ColA::at(xl, y)];  // written by this thread above
      t = cmul(pv[i], t);
      keep[2 * i] = pv[i].x;
      keep[2 * i + 1] = pv[i].y;
    }
    tmem_st16(tm + 32 + 2 * i0, keep);
  }
  tmem_wait_st();
  __syncthreads();
  EPIE_PHASE(1);
  fft_all<N, false, NT, WC, false, ColA>(slab, tw);
  EPIE_PHASE(2);

  // max |O_old|^2 over the patch: FP32 comparisons pick the element (lanes,
  // then warps); its square is formed in FP64 for the cluster-wide maximum
  omv = warp_argmax_f(om, omv);
  float *redf = reinterpret_cast<float *>(red + 2);  // per-warp candidates (re, im, |.|^2)
  if (lane == 0) {
    redf[3 * warp] = omv.x;
    redf[3 * warp + 1] = omv.y;
    redf[3 * warp + 2] = omv.x * omv.x + omv.y * omv.y;
  }
  __syncthreads();
  if (warp == 0) {
    float2 c = make_float2(0.f, 0.f);
    float q = -1.f;
    if (lane < NW) {
      c = make_float2(redf[3 * lane], redf[3 * lane + 1]);
      q = redf[3 * lane + 2];
    }
    c = warp_argmax_f(q, c);
    if (lane == 0) red[0] = static_cast<double>(c.x) * c.x + static_cast<double>(c.y) * c.y;
  }
  double omax = 0.0;

  if constexpr (CL > 1) {
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();  // column transforms and red[0] of every CTA visible
    EPIE_PHASE(3);
    constexpr int CH = HR * WC / 2;  // float4 per (peer, this CTA) block
    float4 t4[E / 2];
#pragma unroll
    for (int i = 0; i < E / 2; ++i) {
      const int m = tid + i * NT, q = m / CH, off = m % CH;
      const float4 *src = reinterpret_cast<const float4 *>(cluster.map_shared_rank(slab, q));
      t4[i] = src[crank * CH + off];
    }
    // one remote load per lane of warp 0: lane q < CL fetches CTA q's patch
    // maximum (FP64 only in this warp: the FP64 pipe is narrow)
    double om_all = 0.0;
    if (warp == 0) {
      om_all = lane < CL ? *cluster.map_shared_rank(red, lane) : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) om_all = fmax(om_all, __shfl_xor_sync(0xffffffffu, om_all, o));
    }
    EPIE_PHASE(4);
    cluster.sync();  // all remote reads done before the tile is overwritten
#pragma unroll
    for (int i = 0; i < E / 2; ++i) {
      const int m = tid + i * NT, q = m / CH, off = m % CH;
      const int e0 = 2 * off, yl = e0 / WC, x = q * WC + e0 % WC;
      slab[RowB::at(yl, x)] = make_float2(t4[i].x, t4[i].y);
      slab[RowB::at(yl, x + 1)] = make_float2(t4[i].z, t4[i].w);
    }
    omax = om_all;
    __syncthreads();
    EPIE_PHASE(5);
  } else {
    __syncthreads();  // red[0] written by thread 0
    if (tid == 0) omax = red[0];
  }

  // ---------------------------------------------------------------- phase 2
  bool ok = mbar_wait_bounded(bar, 0, wait_ns);
  if (!ok) atomicOr(a.err_flag, FLAG_TMA_TIMEOUT);
  ok = __all_sync(0xffffffffu, ok);  // warp-uniform: phase 3 reads TMEM warp-collectively
  float isum_t = 0.f, isum_c = 0.f;  // two-sum of I over this thread's tile elements
  if (!a.amp) {
    // intensity tile -> float max(I - dark, 0), in place: the raw tile sits
    // at the top of the float tile, so every raw value is read (and the dark
    // field fetched with one latency) before any float is written
    constexpr int EI = HR * N / NT;
    float iv[EI];
#pragma unroll
    for (int i = 0; i < EI; ++i) iv[i] = ival(iraw[tid + i * NT]);
    if (a.dark) {
      const float *dk = a.dark + crank * HR * N;
#pragma unroll
      for (int i = 0; i < EI; ++i) iv[i] -= __ldg(dk + tid + i * NT);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < EI; ++i) {
      const float I = fmaxf(iv[i], 0.f);
      two_sum_add(isum_t, isum_c, I);
      itile[tid + i * NT] = sqrtf(I);
    }
    // the first row pass's barrier orders these writes before the modulus
  }
  ModReplace<N> mod{itile, 0.f};
  EPIE_PHASE(6);
  fft_roundtrip_rows<N, NT, HR, RowB>(slab, tw, mod);
  EPIE_PHASE(7);
  {
    // FP32 over a thread's elements, error-free (two-sum) FP32 trees over the
    // warp, FP64 across warps, CTAs and frames
    float *rede = reinterpret_cast<float *>(red + 2);
    float eh = mod.e, el = 0.f, sh = isum_t, sl = isum_c;
    warp_two_sum(eh, el);
    warp_two_sum(sh, sl);
    if (lane == 0) reinterpret_cast<float4 *>(rede)[warp] = make_float4(eh, el, sh, sl);
    __syncthreads();
    if (warp == 0) {
      double es = 0.0, ss = 0.0;
      if (lane < NW) {
        const float4 t4 = reinterpret_cast<const float4 *>(rede)[lane];
        es = two_sum_value(t4.x, t4.y);
        ss = two_sum_value(t4.z, t4.w);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        es += __shfl_xor_sync(0xffffffffu, es, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
      }
      if (lane == 0) {
        a.err_part[static_cast<size_t>(f) * a.err_stride + crank] = es;
        a.isum_part[static_cast<size_t>(f) * a.err_stride + crank] =
            a.amp ? (crank == 0 ? a.amp_isum[f] : 0.0) : ss;
        // the update strengths, once per CTA (FP64 maxima, FP32 divisions:
        // the FP64 pipe is narrow); the error sums above are consumed, so
        // their slots carry the strengths to every thread (the next barrier
        // comes before phase 3 reads them)
        const double pm = __longlong_as_double(static_cast<long long>(*a.pmax2));
        const double om_used = a.omax2_global ? *a.omax2_global : omax;
        const float pmf = static_cast<float>(pm), omf = static_cast<float>(om_used);
        rede[0] = pm > 0.0 ? a.alpha / pmf : 0.f;
        rede[1] = om_used > 0.0 ? a.beta / omf : 0.f;
        rede[2] = pm > 0.0 ? 1.0f / pmf : 0.f;
      }
    }
  }
  EPIE_PHASE(8);

  if constexpr (CL > 1) {
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();
    EPIE_PHASE(9);
    float2 t2[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int idx = tid + i * NT, y = idx / WC, xl = idx % WC;
      const float2 *src = cluster.map_shared_rank(slab, y / HR);
      t2[i] = src[RowB::at(y % HR, crank * WC + xl)];
    }
  EPIE_PHASE(10);
    cluster.sync();
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int idx = tid + i * NT, y = idx / WC, xl = idx % WC;
      slab[ColA::at(xl, y)] = t2[i];
    }
    __syncthreads();
  EPIE_PHASE(11);
  }

  // ---------------------------------------------------------------- phase 3
  fft_all<N, true, NT, WC, false, ColA>(slab, tw);
  EPIE_PHASE(12);

  const float *strength = reinterpret_cast<const float *>(red + 2);
  const float ao = strength[0], bp = strength[1];
  float2 *part = a.probe_part + static_cast<size_t>(member) * N * N + crank * WC;
  if (ok && a.accO == nullptr) {
#pragma unroll
    for (int i0 = 0; i0 < E; i0 += EB) {
      // the object patch and probe values kept in tensor memory in phase 1
      float ko[2 * EB], kp[2 * EB];
      tmem_ld16(tm + 2 * i0, ko);
      tmem_ld16(tm + 32 + 2 * i0, kp);
      tmem_wait_ld();
      float2 pv[EB], ov[EB];
#pragma unroll
      for (int i = 0; i < EB; ++i) {
        pv[i] = make_float2(kp[2 * i], kp[2 * i + 1]);
        ov[i] = make_float2(ko[2 * i], ko[2 * i + 1]);
      }
#pragma unroll
      for (int i = 0; i < EB; ++i) {
        const int idx = tid + (i0 + i) * NT, y = idx / WC, xl = idx % WC;
        const float2 psi1 = slab[ColA::at(xl, y)];
        const float2 d = psub(psi1, cmul(pv[i], ov[i]));
        const float2 uo = cmulc(pv[i], d);  // conj(P) Delta
        const float2 up = cmulc(ov[i], d);  // conj(O_old) Delta
        // paired-FP32 scalings (each lane rounds as the scalar fmaf / multiply)
        EPIE_ST_O(Obase + y * orow + xl, __ffma2_rn(make_float2(ao, ao), uo, ov[i]));
        part[y * N + xl] = __fmul2_rn(up, make_float2(bp, bp));
      }
    }
  } else if (ok) {
    // mini-batch: patches of a batch may overlap; the object moves once per
    // batch by the count-normalised sum, applied by a separate kernel
    const float inv_pm = strength[2];
    const size_t obase = static_cast<size_t>(py) * orow + px + crank * WC;
    float ko[2 * EB], kp[2 * EB];  // a batch of kept object / probe values
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int idx = tid + i * NT, y = idx / WC, xl = idx % WC;
      if (i % EB == 0) {
        tmem_ld16(tm + 2 * i, ko);
        tmem_ld16(tm + 32 + 2 * i, kp);
        tmem_wait_ld();
      }
      const float2 psi1 = slab[ColA::at(xl, y)];
      const float2 p = make_float2(kp[2 * (i % EB)], kp[2 * (i % EB) + 1]);
      const float2 o = make_float2(ko[2 * (i % EB)], ko[2 * (i % EB) + 1]);
      const float2 d = csub(psi1, cmul(p, o));
      const float2 uo = cscale(cmulc(p, d), inv_pm);
      const size_t oi = obase + y * orow + xl;
      atomicAdd(a.accO + oi, uo);  // one paired (8-byte) atomic
      atomicAdd(a.cnt + oi, 1);
      part[y * N + xl] = cscale(cmulc(o, d), bp);
    }
  } else {
    // the copy never arrived: give it one more bounded wait before exiting
    mbar_wait_bounded(bar, 0, wait_ns < 100000000ull ? wait_ns : 100000000ull);
  }
#undef EPIE_LD_O
#undef EPIE_ST_O
  // every thread's tensor-memory reads are done before warp 0 frees it
  tc_fence_before();
  __syncthreads();
  EPIE_PHASE(13);
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tm_base, C::TM_COLS);
  }
}

template <int N, int CL, int NT, typename IT>
cudaError_t launch_fused_t(const GroupArgs &a, cudaStream_t st) {
  using C = FusedCfg<N, CL, NT, IT>;
  auto kern = epie_fused_kernel<N, CL, NT, IT>;
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!configured[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(C::SMEM));
    if (e != cudaSuccess) return e;
    // prefer the whole unified L1 / shared-memory array as shared memory
    // (2 resident CTAs of this size)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    if (CL > 8) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    // A TMEM allocation blocks until columns are free, and CTAs of a cluster
    // wait for each other, so every CTA that can be resident on an SM must
    // find its columns at once: at most 512 in total.  Any step kernel is
    // held to 2 resident CTAs of <= 256 columns, or 1 of <= 512 (the tcgen05
    // GEMM's shared memory keeps it off SMs that hold a step kernel).
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, C::SMEM);
    if (e != cudaSuccess) return e;
    if (occ < 1 || occ * C::TM_COLS > 512 || (occ > 1 && C::TM_COLS > 256))
      return cudaErrorInvalidConfiguration;
    configured[dev] = true;
  }
  if (a.n_members <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(a.n_members * CL), 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int na = 0;
  attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[na].val.programmaticStreamSerializationAllowed = 1;
  ++na;
  if (CL > 1) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = CL;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace epie
