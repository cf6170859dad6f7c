// epie_aux.cu -- kernels around the fused ePIE step: live ingest (DC shift),
// the per-group probe reduction with its FP64 max|P|^2, FP64 maxima and the
// sweep-error reduction, and the pieces of the plain unfused path
// (gather / modulus / update) that runs the same step with cuFFT in between.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/epie.h"
#include "epie_fft.cuh"
#include "epie_ingest.cuh"
#include "epie_internal.h"

namespace epie {

namespace {

// bits of a non-negative double order like the double itself
__device__ __forceinline__ void atomic_max_pos_double(unsigned long long *slot, double v) {
  atomicMax(slot, static_cast<unsigned long long>(__double_as_longlong(v)));
}

// |v|^2 in FP64 of the block's element of largest |v|^2 (FP32 comparisons
// pick the element: lanes, then warps), valid in thread 0.  The FP64 square
// is formed once per block: the FP64 pipe is narrow.
template <int NT>
__device__ double block_abs2_max(float q, float2 v, float4 *sh) {
  v = warp_argmax_f(q, v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = make_float4(v.x, v.y, v.x * v.x + v.y * v.y, 0.f);
  __syncthreads();
  double m = 0.0;
  if (threadIdx.x == 0) {
    float4 best = sh[0];
    for (int w = 1; w < NT / 32; ++w)
      if (sh[w].z > best.z) best = sh[w];
    m = static_cast<double>(best.x) * best.x + static_cast<double>(best.y) * best.y;
  }
  __syncthreads();
  return m;
}

// ---------------------------------------------------------------- ingest

// DC-centred detector frame -> FFT order: dst[ky][kx] = src[(ky+N/2)%N][(kx+N/2)%N].
// Rows hold N*esize bytes (a multiple of 16); the half-row rotation moves
// whole 16-byte chunks, so each thread copies one uint4.
__global__ void ingest_kernel(const uint4 *__restrict__ src, uint4 *__restrict__ dst, int n,
                              int N, int chunks_per_row) {
  const long long total = static_cast<long long>(n) * N * chunks_per_row;
  for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(t % chunks_per_row);
    const long long rowid = t / chunks_per_row;
    const int ky = static_cast<int>(rowid % N);
    const long long f = rowid / N;
    const int sy = (ky + N / 2) % N;
    const int sc = (c + chunks_per_row / 2) % chunks_per_row;
    dst[t] = src[(f * N + sy) * chunks_per_row + sc];
  }
}

__global__ void dark_ingest_kernel(const float *__restrict__ src, float *__restrict__ dst, int N) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * N) return;
  const int ky = t / N, kx = t % N;
  dst[t] = src[((ky + N / 2) % N) * N + (kx + N / 2) % N];
}

// ---------------------------------------------------------------- probe

// P += scale * sum_{m < n_members} part[m], then the FP64 max|P|^2 of the
// new probe (FP32 comparison picks the element).  A block of 32 x PR_ROWS
// threads covers 64 complex elements (two per thread, 16-byte loads); thread
// row r sums members r, r + PR_ROWS, ... in order and the row sums are added
// in row order, so the result does not depend on scheduling.  The partials
// are read once, with the streaming hint, so their lines leave L2 before the
// object's.  A thread issues the loads of 4 of its members at a time, the
// last batch predicated past the last member.
#ifndef EPIE_PROBE_ROWS
#define EPIE_PROBE_ROWS 8
#endif
constexpr int PR_ROWS = EPIE_PROBE_ROWS, PR_THREADS = 32 * PR_ROWS;
__global__ void __launch_bounds__(PR_THREADS, 5) probe_reduce_kernel(
    float2 *__restrict__ P, const float2 *__restrict__ part, int n_members, int K, float scale,
    unsigned long long *pmax2_next, const int32_t *gstart, int group, int mean) {
  __shared__ float4 acc_sh[PR_ROWS][32];
  __shared__ float4 sh[PR_THREADS / 32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (gstart) {  // group size from the device table
    n_members = gstart[group + 1] - gstart[group];
    scale = mean ? 1.0f / static_cast<float>(n_members) : 1.0f;
  }
  grid_dependency_wait();  // the partials of the preceding step kernel
  grid_dependents_launch();
  float best = -1.f;
  float2 bv = make_float2(0.f, 0.f);
  auto ld = [&](int m, int i) {
    return __ldcs(reinterpret_cast<const float4 *>(part + static_cast<size_t>(m) * K + i));
  };
  for (int base = blockIdx.x * 64; base < K; base += gridDim.x * 64) {
    const int i = base + 2 * tx;  // K is a multiple of 64
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int m0 = ty; m0 < n_members; m0 += 4 * PR_ROWS) {
      float4 a[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        a[k] = m0 + k * PR_ROWS < n_members ? ld(m0 + k * PR_ROWS, i) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (m0 + k * PR_ROWS < n_members) {  // members in order; none added past the last
          acc.x += a[k].x; acc.y += a[k].y; acc.z += a[k].z; acc.w += a[k].w;
        }
      }
    }
    acc_sh[ty][tx] = acc;
    __syncthreads();
    if (ty == 0) {
      float4 t = acc_sh[0][tx];
#pragma unroll
      for (int r = 1; r < PR_ROWS; ++r) {
        const float4 u = acc_sh[r][tx];
        t.x += u.x; t.y += u.y; t.z += u.z; t.w += u.w;
      }
      float4 p = *reinterpret_cast<float4 *>(P + i);
      p.x = fmaf(scale, t.x, p.x);
      p.y = fmaf(scale, t.y, p.y);
      p.z = fmaf(scale, t.z, p.z);
      p.w = fmaf(scale, t.w, p.w);
      *reinterpret_cast<float4 *>(P + i) = p;
      const float q0 = p.x * p.x + p.y * p.y, q1 = p.z * p.z + p.w * p.w;
      if (q0 > best) { best = q0; bv = make_float2(p.x, p.y); }
      if (q1 > best) { best = q1; bv = make_float2(p.z, p.w); }
    }
    __syncthreads();
  }
  const double d = block_abs2_max<PR_THREADS>(best, bv, sh);
  if (threadIdx.x == 0) atomic_max_pos_double(pmax2_next, d);
}

template <int NT>
__global__ void __launch_bounds__(NT) abs2_max_kernel(const float2 *__restrict__ a, long long n,
                                                      unsigned long long *out) {
  __shared__ float4 sh[NT / 32];
  float best = -1.f;
  float2 bv = make_float2(0.f, 0.f);
  for (long long i = blockIdx.x * static_cast<long long>(NT) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * NT) {
    const float2 p = a[i];
    const float q = p.x * p.x + p.y * p.y;
    if (q > best) { best = q; bv = p; }
  }
  const double d = block_abs2_max<NT>(best, bv, sh);
  if (threadIdx.x == 0) atomic_max_pos_double(out, d);
}

__global__ void bits_to_double_kernel(const unsigned long long *bits, double *out) {
  *out = __longlong_as_double(static_cast<long long>(*bits));
}

// ---------------------------------------------------------------- sweep error

// One block: thread t sums frames t, t+NT, ... (slots in order), then a
// fixed tree over threads.  E = sum e / sum s (0 when sum s = 0).
template <int NT>
__global__ void __launch_bounds__(NT) error_reduce_kernel(const double *__restrict__ e,
                                                          const double *__restrict__ s,
                                                          int n_frames, int stride,
                                                          double *out) {
  __shared__ double se[NT], ss[NT];
  double a = 0.0, b = 0.0;
  for (int f = threadIdx.x; f < n_frames; f += NT)
    for (int c = 0; c < stride; ++c) {
      a += e[static_cast<size_t>(f) * stride + c];
      b += s[static_cast<size_t>(f) * stride + c];
    }
  se[threadIdx.x] = a;
  ss[threadIdx.x] = b;
  __syncthreads();
  for (int h = NT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      se[threadIdx.x] += se[threadIdx.x + h];
      ss[threadIdx.x] += ss[threadIdx.x + h];
    }
    __syncthreads();
  }
  // 0 for an empty sweep; a non-finite sum gives a non-finite error
  if (threadIdx.x == 0) *out = ss[0] == 0.0 ? 0.0 : se[0] / ss[0];
}

// Stage 1 of the sweep error: block b sums frames [b per, (b + 1) per) (thread
// t takes frames b per + t, + 256, ..., all slots of each in order), then a
// fixed tree over the threads; writes (sum e, sum s) of its range.
__global__ void __launch_bounds__(256) error_block_kernel(const double *__restrict__ e,
                                                          const double *__restrict__ s,
                                                          int n_frames, int stride, int per,
                                                          double *__restrict__ blocks) {
  __shared__ double se[256], ss[256];
  const int f0 = blockIdx.x * per, f1 = min(n_frames, f0 + per);
  double a = 0.0, b = 0.0;
  for (int f = f0 + threadIdx.x; f < f1; f += 256)
    for (int c = 0; c < stride; ++c) {
      a += e[static_cast<size_t>(f) * stride + c];
      b += s[static_cast<size_t>(f) * stride + c];
    }
  se[threadIdx.x] = a;
  ss[threadIdx.x] = b;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      se[threadIdx.x] += se[threadIdx.x + h];
      ss[threadIdx.x] += ss[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    blocks[2 * blockIdx.x] = se[0];
    blocks[2 * blockIdx.x + 1] = ss[0];
  }
}

// Stage 2: E = sum e / sum s over the ERR_BLOCKS block sums (fixed tree); 0
// for an empty sweep, non-finite when a sum is
__global__ void __launch_bounds__(ERR_BLOCKS) error_final_kernel(const double *__restrict__ blocks,
                                                                 double *out) {
  __shared__ double se[ERR_BLOCKS], ss[ERR_BLOCKS];
  se[threadIdx.x] = blocks[2 * threadIdx.x];
  ss[threadIdx.x] = blocks[2 * threadIdx.x + 1];
  __syncthreads();
  for (int h = ERR_BLOCKS / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      se[threadIdx.x] += se[threadIdx.x + h];
      ss[threadIdx.x] += ss[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = ss[0] == 0.0 ? 0.0 : se[0] / ss[0];
}

// ---------------------------------------------------------------- plain path

// psi[m] = P . O_j for every member; max|O_j|^2 per member (bits)
// psi = P . O_j per member, or (hi set) psi split into bf16 hi = bf16(psi)
// and lo = bf16(psi - hi) for the tensor-core DFT (lo may be null)
__global__ void plain_gather_kernel(GroupArgs a, int N, float2 *__restrict__ psi,
                                    unsigned long long *__restrict__ omax_bits,
                                    __nv_bfloat162 *__restrict__ hi, __nv_bfloat162 *__restrict__ lo) {
  __shared__ float4 sh[8];
  const int m = blockIdx.y, K = N * N;
  const int f = a.members[m];
  const int py = a.pos[2 * f], px = a.pos[2 * f + 1];
  float best = -1.f;
  float2 bv = make_float2(0.f, 0.f);
  for (int i = blockIdx.x * 256 + threadIdx.x; i < K; i += gridDim.x * 256) {
    const int y = i / N, x = i % N;
    const float2 o = a.O[static_cast<size_t>(py + y) * a.W + px + x];
    const float2 v = cmul(a.P[i], o);
    const size_t t = static_cast<size_t>(m) * K + i;
    if (hi) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
      hi[t] = h;
      if (lo) lo[t] = __floats2bfloat162_rn(v.x - __low2float(h), v.y - __high2float(h));
    } else {
      psi[t] = v;
    }
    const float q = o.x * o.x + o.y * o.y;
    if (q > best) { best = q; bv = o; }
  }
  const double d = block_abs2_max<256>(best, bv, sh);
  if (threadIdx.x == 0) atomic_max_pos_double(omax_bits + m, d);
}

// modulus replacement on the cuFFT spectrum (1/N^2 folded in); 256 threads x
// 4 elements per block, per-block error partials
template <typename IT>
__global__ void plain_modulus_kernel(GroupArgs a, int N, float2 *__restrict__ Psi) {
  __shared__ float4 red[8];
  const int m = blockIdx.y, K = N * N;
  const int f = a.members[m];
  const IT *I = static_cast<const IT *>(a.frames) + static_cast<size_t>(f) * K;
  const float invK = 1.0f / (static_cast<float>(N) * static_cast<float>(N));
  float e = 0.f, s = 0.f;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int k = blockIdx.x * 1024 + r * 256 + threadIdx.x;
    float In = ival(I[k]);
    if (a.dark) In -= a.dark[k];
    In = fmaxf(In, 0.f);
    const float sq = sqrtf(In);
    float2 v = Psi[static_cast<size_t>(m) * K + k];
    const float a2 = v.x * v.x + v.y * v.y;
    float amp;
    if (a2 > 0.f) {
      const float ia = rsqrtf(a2);
      amp = a2 * ia;
      v = cscale(v, sq * ia * invK);
    } else {
      amp = 0.f;
      v = make_float2(sq * invK, 0.f);
    }
    Psi[static_cast<size_t>(m) * K + k] = v;
    const float d = amp - sq;
    e = fmaf(d, d, e);
    s += In;
  }
  // FP32 per thread, error-free FP32 trees per warp, FP64 across warps (one thread)
  float el = 0.f, sl = 0.f;
  warp_two_sum(e, el);
  warp_two_sum(s, sl);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_float4(e, el, s, sl);
  __syncthreads();
  if (threadIdx.x == 0) {
    double te = 0.0, ts = 0.0;
    for (int w = 0; w < 8; ++w) {
      te += two_sum_value(red[w].x, red[w].y);
      ts += two_sum_value(red[w].z, red[w].w);
    }
    a.err_part[static_cast<size_t>(f) * a.err_stride + blockIdx.x] = te;
    a.isum_part[static_cast<size_t>(f) * a.err_stride + blockIdx.x] = ts;
  }
}

// (alpha_eff / max|P|^2, beta / max|O|^2) of a member, once per block
// (thread 0; FP64 maxima, FP32 divisions) and handed to every thread
// through shared memory
__device__ float2 block_strengths(const GroupArgs &a, unsigned long long omax_bits, float alpha_eff) {
  __shared__ float2 st;
  if (threadIdx.x == 0) {
    const double pm = __longlong_as_double(static_cast<long long>(*a.pmax2));
    const double om = a.omax2_global ? *a.omax2_global
                                     : __longlong_as_double(static_cast<long long>(omax_bits));
    st = make_float2(pm > 0.0 ? alpha_eff / static_cast<float>(pm) : 0.f,
                     om > 0.0 ? a.beta / static_cast<float>(om) : 0.f);
  }
  __syncthreads();
  return st;
}

// O patch update and probe partial from psi' (= inverse cuFFT output)
__global__ void plain_update_kernel(GroupArgs a, int N, const float2 *__restrict__ psi1,
                                    const unsigned long long *__restrict__ omax_bits) {
  const int m = blockIdx.y, K = N * N;
  const int f = a.members[m];
  const int py = a.pos[2 * f], px = a.pos[2 * f + 1];
  const float2 st = block_strengths(a, omax_bits[m], a.alpha);
  const float ao = st.x, bp = st.y;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && a.pmax2_clear) *a.pmax2_clear = 0ull;
  for (int i = blockIdx.x * 256 + threadIdx.x; i < K; i += gridDim.x * 256) {
    const int y = i / N, x = i % N;
    float2 *op = a.O + static_cast<size_t>(py + y) * a.W + px + x;
    const float2 o = *op, p = a.P[i];
    const float2 d = csub(psi1[static_cast<size_t>(m) * K + i], cmul(p, o));
    const float2 uo = cmulc(p, d), up = cmulc(o, d);
    *op = make_float2(fmaf(ao, uo.x, o.x), fmaf(ao, uo.y, o.y));
    a.probe_part[static_cast<size_t>(m) * K + i] = cscale(up, bp);
  }
}

// ---------------------------------------------------------------- mini-batch

// accumulate conj(P) Delta / max|P|^2 into accO and the coverage count
// (overlapping patches: float atomics, order-dependent rounding only)
__global__ void mb_accumulate_kernel(GroupArgs a, int N, const float2 *__restrict__ psi1,
                                     const unsigned long long *__restrict__ omax_bits,
                                     float2 *__restrict__ accO, int *__restrict__ cnt) {
  const int m = blockIdx.y, K = N * N;
  const int f = a.members[m];
  const int py = a.pos[2 * f], px = a.pos[2 * f + 1];
  const float2 st = block_strengths(a, omax_bits[m], 1.0f);
  const float ao = st.x, bp = st.y;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && a.pmax2_clear) *a.pmax2_clear = 0ull;
  for (int i = blockIdx.x * 256 + threadIdx.x; i < K; i += gridDim.x * 256) {
    const int y = i / N, x = i % N;
    const size_t oi = static_cast<size_t>(py + y) * a.W + px + x;
    const float2 o = a.O[oi], p = a.P[i];
    const float2 d = csub(psi1[static_cast<size_t>(m) * K + i], cmul(p, o));
    const float2 uo = cscale(cmulc(p, d), ao), up = cmulc(o, d);
    atomicAdd(accO + oi, uo);  // one paired (8-byte) atomic
    atomicAdd(cnt + oi, 1);
    a.probe_part[static_cast<size_t>(m) * K + i] = cscale(up, bp);
  }
}

// O += alpha accO / cnt where cnt > 0; clears the accumulators
__global__ void mb_apply_kernel(float2 *__restrict__ O, float2 *__restrict__ accO,
                                int *__restrict__ cnt, long long n, float alpha) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int c = cnt[i];
    if (c > 0) {
      const float2 u = accO[i];
      const float s = alpha / static_cast<float>(c);
      float2 o = O[i];
      o.x = fmaf(s, u.x, o.x);
      o.y = fmaf(s, u.y, o.y);
      O[i] = o;
      accO[i] = make_float2(0.f, 0.f);
      cnt[i] = 0;
    }
  }
}

// The same over the batch's footprint only: every pixel of every member's
// N x N patch.  A pixel covered by several patches is visited several times;
// the visitor that takes its count (atomic exchange with 0) applies and
// clears it, the others find 0.  Member ids come from the group table
// (members of group `group` when gstart is set).
__global__ void mb_apply_local_kernel(float2 *__restrict__ O, float2 *__restrict__ accO,
                                      int *__restrict__ cnt, int W, const int32_t *__restrict__ pos,
                                      const int32_t *__restrict__ members, int n_members,
                                      const int32_t *__restrict__ gstart, int group, int N,
                                      float alpha) {
  if (gstart) {
    members += gstart[group];
    n_members = gstart[group + 1] - gstart[group];
  }
  const int m = blockIdx.y;
  if (m >= n_members) return;
  const int f = members[m];
  const int py = pos[2 * f], px = pos[2 * f + 1];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N * N; i += gridDim.x * blockDim.x) {
    const size_t oi = static_cast<size_t>(py + i / N) * W + px + i % N;
    const int c = atomicExch(cnt + oi, 0);
    if (c > 0) {
      const float2 u = accO[oi];
      const float s = alpha / static_cast<float>(c);
      float2 o = O[oi];
      o.x = fmaf(s, u.x, o.x);
      o.y = fmaf(s, u.y, o.y);
      O[oi] = o;
      accO[oi] = make_float2(0.f, 0.f);
    }
  }
}

__global__ void fill_kernel(float2 *__restrict__ p, long long n, float2 v) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    p[i] = v;
}

int grid_for(long long n, int nt, int cap) {
  long long g = (n + nt - 1) / nt;
  if (g > cap) g = cap;
  return g < 1 ? 1 : static_cast<int>(g);
}

}  // namespace

cudaError_t launch_ingest(const void *raw, void *dst, int n, int N, int esize, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int cpr = N * esize / 16;
  const long long total = static_cast<long long>(n) * N * cpr;
  ingest_kernel<<<grid_for(total, 256, 152 * 16), 256, 0, st>>>(
      static_cast<const uint4 *>(raw), static_cast<uint4 *>(dst), n, N, cpr);
  return cudaGetLastError();
}

namespace {
__global__ void average_kernel(const float2 *const *__restrict__ src, int k, float2 *out,
                               long long n) {
  const float inv = 1.0f / static_cast<float>(k);
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < k; ++q) acc = cadd(acc, src[q][i]);
    out[i] = cscale(acc, inv);
  }
}
}  // namespace

cudaError_t launch_average(const float2 *const *src, int k, float2 *out, long long n,
                           cudaStream_t st) {
  average_kernel<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(src, k, out, n);
  return cudaGetLastError();
}

cudaError_t launch_fill(float2 *p, long long n, float2 v, cudaStream_t st) {
  fill_kernel<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(p, n, v);
  return cudaGetLastError();
}

namespace {
// Measured amplitude of frames [f0, f0 + n) in FFT order: amp = sqrt(max(I -
// dark, 0)), and the frame's sum of max(I - dark, 0) (error-free FP32 per
// thread, FP64 across threads).  One block per frame; each thread takes
// chunks of 8 consecutive elements, loads up to AI_U chunks as 16-byte
// vectors before converting any, and writes each chunk as two float4.  Each
// thread sums a fixed set of elements and the block adds the thread sums in
// a fixed order, so the sums do not depend on scheduling.
constexpr int AI_NT = 512, AI_U = 4;
template <typename IT>
__global__ void __launch_bounds__(AI_NT) amp_ingest_kernel(const IT *__restrict__ frames,
                                                          const float *__restrict__ dark,
                                                          float *__restrict__ amp,
                                                          double *__restrict__ isum, int f0, int K) {
  __shared__ double sh[AI_NT];
  const size_t base = static_cast<size_t>(f0 + blockIdx.x) * K;
  const IT *fr = frames + base;
  float *out = amp + base;
  const int t = threadIdx.x, nc = K >> 3;  // K is a multiple of 8
  float s = 0.f, cc = 0.f;  // error-free FP32 sum (the FP64 pipe is narrow)
  for (int g = 0; g < nc; g += AI_NT * AI_U) {
    Raw8<IT> r[AI_U];
#pragma unroll
    for (int u = 0; u < AI_U; ++u) {
      const int c = g + t + AI_NT * u;
      if (c < nc) r[u].load(fr + 8 * static_cast<size_t>(c));
    }
#pragma unroll
    for (int u = 0; u < AI_U; ++u) {
      const int c = g + t + AI_NT * u;
      if (c < nc) {
        float d[8], v[8];
        dark8(dark ? dark + 8 * static_cast<size_t>(c) : nullptr, d);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          v[i] = clamp_sub(r[u].at(i), d[i]);
          two_sum_add(s, cc, v[i]);
          v[i] = sqrtf(v[i]);
        }
        float4 *o = reinterpret_cast<float4 *>(out + 8 * static_cast<size_t>(c));
        o[0] = make_float4(v[0], v[1], v[2], v[3]);
        o[1] = make_float4(v[4], v[5], v[6], v[7]);
      }
    }
  }
  sh[t] = two_sum_value(s, cc);
  __syncthreads();
  for (int w = AI_NT / 2; w > 0; w >>= 1) {
    if (t < w) sh[t] += sh[t + w];
    __syncthreads();
  }
  if (t == 0) isum[f0 + blockIdx.x] = sh[0];
}
}  // namespace

cudaError_t launch_amp_ingest(const void *frames, int itype, const float *dark, float *amp,
                              double *isum, int f0, int n, int N, int cl, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  // the 1-CTA 128^2, the 256^2 and the 512^2 step kernels read their own tile
  // layouts (epie_fused_128.cu, epie_fused_256.cu, epie_fused_512.cu)
  if (N == 128 && fused_ctas_per_frame(128, cl) == 1)
    return launch_amp_ingest_128(frames, itype, dark, amp, isum, f0, n, st);
  if (N == 256) return launch_amp_ingest_256(frames, itype, dark, amp, isum, f0, n, st);
  if (N == 512) return launch_amp_ingest_512(frames, itype, dark, amp, isum, f0, n, st);
  const int K = N * N;
  if (itype == EPIE_U16)
    amp_ingest_kernel<<<n, AI_NT, 0, st>>>(static_cast<const uint16_t *>(frames), dark, amp, isum,
                                          f0, K);
  else if (itype == EPIE_F16)
    amp_ingest_kernel<<<n, AI_NT, 0, st>>>(static_cast<const __half *>(frames), dark, amp, isum,
                                          f0, K);
  else
    amp_ingest_kernel<<<n, AI_NT, 0, st>>>(static_cast<const float *>(frames), dark, amp, isum, f0,
                                          K);
  return cudaGetLastError();
}

cudaError_t launch_dark_ingest(const float *raw, float *dst, int N, cudaStream_t st) {
  dark_ingest_kernel<<<(N * N + 255) / 256, 256, 0, st>>>(raw, dst, N);
  return cudaGetLastError();
}

cudaError_t launch_probe_reduce(float2 *P, const float2 *part, int n_members, int N, float scale,
                                unsigned long long *pmax2_next, cudaStream_t st) {
  const int K = N * N;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid_for(K, 64, 152 * 8), 1, 1);
  cfg.blockDim = dim3(PR_THREADS, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, probe_reduce_kernel, P, part, n_members, K, scale, pmax2_next,
                            static_cast<const int32_t *>(nullptr), 0, 0);
}

cudaError_t launch_probe_reduce_table(float2 *P, const float2 *part, const int32_t *gstart,
                                      int group, int mean, int N, unsigned long long *pmax2_next,
                                      cudaStream_t st) {
  const int K = N * N;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid_for(K, 64, 152 * 8), 1, 1);
  cfg.blockDim = dim3(PR_THREADS, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, probe_reduce_kernel, P, part, 0, K, 1.0f, pmax2_next, gstart,
                            group, mean);
}

namespace {
__global__ void copy_u64_kernel(const unsigned long long *src, unsigned long long *dst) {
  *dst = *src;
}
}  // namespace

cudaError_t launch_copy_u64(const unsigned long long *src, unsigned long long *dst,
                            cudaStream_t st) {
  copy_u64_kernel<<<1, 1, 0, st>>>(src, dst);
  return cudaGetLastError();
}

cudaError_t launch_probe_max(const float2 *P, int K, unsigned long long *pmax2, cudaStream_t st) {
  abs2_max_kernel<256><<<grid_for(K, 256, 152 * 2), 256, 0, st>>>(P, K, pmax2);
  return cudaGetLastError();
}

cudaError_t launch_object_max(const float2 *O, long long n, double *out, unsigned long long *tmp,
                              cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(tmp, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  abs2_max_kernel<256><<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(O, n, tmp);
  bits_to_double_kernel<<<1, 1, 0, st>>>(tmp, out);
  return cudaGetLastError();
}

cudaError_t launch_error_reduce(const double *err_part, const double *isum_part, int n_frames,
                                int stride, double *out, double *blocks, cudaStream_t st) {
  // two fixed-order stages: ERR_BLOCKS blocks over contiguous frame ranges,
  // then one block over their sums (FP64 adds spread over many SMs: the FP64
  // pipe of a single SM made one block the bottleneck)
  const int per = (n_frames + ERR_BLOCKS - 1) / ERR_BLOCKS;
  error_block_kernel<<<ERR_BLOCKS, 256, 0, st>>>(err_part, isum_part, n_frames, stride, per,
                                                 blocks);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  error_final_kernel<<<1, ERR_BLOCKS, 0, st>>>(blocks, out);
  return cudaGetLastError();
}

int plain_err_stride(int N) { return N * N / 1024; }

cudaError_t launch_plain_gather(const GroupArgs &a, int N, float2 *psi, double *omax2,
                                cudaStream_t st, void *hi, void *lo) {
  auto *bits = reinterpret_cast<unsigned long long *>(omax2);
  cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(unsigned long long) * a.n_members, st);
  if (e != cudaSuccess) return e;
  dim3 grid(N * N / 1024, a.n_members);
  plain_gather_kernel<<<grid, 256, 0, st>>>(a, N, psi, bits, static_cast<__nv_bfloat162 *>(hi),
                                            static_cast<__nv_bfloat162 *>(lo));
  return cudaGetLastError();
}

cudaError_t launch_plain_modulus(const GroupArgs &a, int N, int itype, float2 *Psi,
                                 cudaStream_t st) {
  dim3 grid(N * N / 1024, a.n_members);
  if (itype == 0) plain_modulus_kernel<uint16_t><<<grid, 256, 0, st>>>(a, N, Psi);
  else if (itype == 1) plain_modulus_kernel<__half><<<grid, 256, 0, st>>>(a, N, Psi);
  else plain_modulus_kernel<float><<<grid, 256, 0, st>>>(a, N, Psi);
  return cudaGetLastError();
}

cudaError_t launch_plain_update(const GroupArgs &a, int N, const float2 *psi1, const double *omax2,
                                cudaStream_t st) {
  dim3 grid(N * N / 1024, a.n_members);
  plain_update_kernel<<<grid, 256, 0, st>>>(a, N, psi1,
                                            reinterpret_cast<const unsigned long long *>(omax2));
  return cudaGetLastError();
}

cudaError_t launch_mb_accumulate(const GroupArgs &a, int N, const float2 *psi1,
                                 const double *omax2, float2 *accO, int *cnt, cudaStream_t st) {
  dim3 grid(N * N / 1024, a.n_members);
  mb_accumulate_kernel<<<grid, 256, 0, st>>>(
      a, N, psi1, reinterpret_cast<const unsigned long long *>(omax2), accO, cnt);
  return cudaGetLastError();
}

cudaError_t launch_mb_apply(float2 *O, float2 *accO, int *cnt, long long n, float alpha,
                            cudaStream_t st) {
  mb_apply_kernel<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(O, accO, cnt, n, alpha);
  return cudaGetLastError();
}

cudaError_t launch_mb_apply_local(float2 *O, float2 *accO, int *cnt, int W, const int32_t *pos,
                                  const int32_t *members, int n_members, const int32_t *gstart,
                                  int group, int N, float alpha, cudaStream_t st) {
  if (n_members <= 0) return cudaSuccess;
  dim3 grid((N * N + 1023) / 1024, n_members);
  mb_apply_local_kernel<<<grid, 256, 0, st>>>(O, accO, cnt, W, pos, members, n_members, gstart,
                                              group, N, alpha);
  return cudaGetLastError();
}

}  // namespace epie
