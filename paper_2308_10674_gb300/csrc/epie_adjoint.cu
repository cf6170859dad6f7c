// epie_adjoint.cu -- amplitude loss and its hand-written adjoint.
//
//   L = sum_j sum_k ( |F(S_dj P . O_j)|(k) - sqrt(I_j(k)) )^2
//
// with S_d P = F^-1[ F P . exp(-2 pi i (ky dy + kx dx)/N) ] a Fourier shift of
// the probe by the sub-pixel offset d_j of position j (frequencies in FFT
// order, k >= N/2 standing for k - N).  The ePIE step of the paper (Sec.
// "ePIE Implementation") is a projection on the set this loss measures the
// distance to; its gradient lets the same forward model be optimised jointly
// over object, probe and positions.  Gradients follow the convention
// dL/dRe + i dL/dIm; where |Psi| = 0 the amplitude's gradient is taken as 0.
//
// One thread-block cluster per position runs four 2-D transforms with the
// frame spread over its CTAs (column blocks <-> row blocks through
// distributed shared memory, as in the fused ePIE kernel):
//   Z = FP . ph   -- F^-1 -->  Ps = S_d P          (row blocks; kept in smem)
//   psi = Ps . O_j -- F -->    Psi                 (column blocks)
//   G = 2 (|Psi| - sqrt I) Psi/|Psi| -- F^H --> g_psi (row blocks)
//   g_O += conj(Ps) g_psi;  g_Ps = conj(O_j) g_psi -- F/K --> gZ (columns)
//   d L/d d = Re sum conj(gZ) Z (-2 pi i k/N);  g_FP += gZ conj(ph)
// Nothing is stored between positions: the far field is recomputed inside the
// kernel.  Object and probe-spectrum gradients accumulate with float atomics
// (summation order not fixed); the loss and the position gradients use
// per-CTA partials reduced in a fixed order.  g_P = K F^-1(g_FP) at the end.
#include <cooperative_groups.h>
#include <cuda_fp16.h>

#include <string>
#include <type_traits>

#include "../../include/epie.h"
#include "epie_fft.cuh"
#include "epie_internal.h"

namespace epie {
std::string &init_error_sink();
}

namespace {

using namespace epie;
namespace cg = cooperative_groups;

constexpr double kPi = 3.14159265358979323846;

template <int N, int CL>
struct AdjCfg {
  static constexpr int WC = N / CL, HR = N / CL, PB = N + N / 16;
  static constexpr int NT = N * N / (CL * 16);
  static constexpr int E = 16;
  static constexpr int NW = NT / 32;
  static constexpr int SLAB = CL == 1 ? N * PB : (N * WC > HR * PB ? N * WC : HR * PB);
  static constexpr size_t OFF_TW = sizeof(float2) * SLAB;
  static constexpr size_t OFF_AUX = OFF_TW + sizeof(float2) * N;  // Ps, row blocks [HR][N]
  static constexpr size_t OFF_RED = OFF_AUX + sizeof(float2) * HR * N;
  static constexpr size_t SMEM = OFF_RED + sizeof(double) * 4 * NW;
};

template <int N, int CL>
using ColA = ColAddr<CL == 1 ? AdjCfg<N, CL>::PB : AdjCfg<N, CL>::WC, CL == 1>;
template <int N, int CL>
using RowB = RowAddr<AdjCfg<N, CL>::PB>;

// FFT frequency of index k (k >= N/2 stands for k - N)
template <int N>
__device__ __forceinline__ float freq(int k) {
  return static_cast<float>(k < N / 2 ? k : k - N);
}

// exp(-2 pi i (fy dy + fx dx) / N)
template <int N>
__device__ __forceinline__ float2 shift_phase(int ky, int kx, float dy, float dx) {
  float s, c;
  sincospif(-2.0f * (freq<N>(ky) * dy + freq<N>(kx) * dx) / static_cast<float>(N), &s, &c);
  return make_float2(c, s);
}

// column blocks [N][WC] -> row blocks [HR][PB] across the cluster
template <int N, int CL>
__device__ __forceinline__ void cols_to_rows(float2 *slab) {
  using C = AdjCfg<N, CL>;
  if constexpr (CL > 1) {
    cg::cluster_group cluster = cg::this_cluster();
    const int crank = static_cast<int>(cluster.block_rank());
    constexpr int CH = C::HR * C::WC / 2;
    float4 t4[C::E / 2];
    cluster.sync();
#pragma unroll
    for (int i = 0; i < C::E / 2; ++i) {
      const int m = threadIdx.x + i * C::NT, q = m / CH, off = m % CH;
      const float4 *src = reinterpret_cast<const float4 *>(cluster.map_shared_rank(slab, q));
      t4[i] = src[crank * CH + off];
    }
    cluster.sync();
#pragma unroll
    for (int i = 0; i < C::E / 2; ++i) {
      const int m = threadIdx.x + i * C::NT, q = m / CH, off = m % CH;
      const int e0 = 2 * off, yl = e0 / C::WC, x = q * C::WC + e0 % C::WC;
      slab[RowB<N, CL>::at(yl, x)] = make_float2(t4[i].x, t4[i].y);
      slab[RowB<N, CL>::at(yl, x + 1)] = make_float2(t4[i].z, t4[i].w);
    }
  }
  __syncthreads();
}

// row blocks -> column blocks across the cluster
template <int N, int CL>
__device__ __forceinline__ void rows_to_cols(float2 *slab) {
  using C = AdjCfg<N, CL>;
  if constexpr (CL > 1) {
    cg::cluster_group cluster = cg::this_cluster();
    const int crank = static_cast<int>(cluster.block_rank());
    float2 t2[C::E];
    cluster.sync();
#pragma unroll
    for (int i = 0; i < C::E; ++i) {
      const int idx = threadIdx.x + i * C::NT, y = idx / C::WC, xl = idx % C::WC;
      const float2 *src = cluster.map_shared_rank(slab, y / C::HR);
      t2[i] = src[RowB<N, CL>::at(y % C::HR, crank * C::WC + xl)];
    }
    cluster.sync();
#pragma unroll
    for (int i = 0; i < C::E; ++i) {
      const int idx = threadIdx.x + i * C::NT, y = idx / C::WC, xl = idx % C::WC;
      slab[ColA<N, CL>::at(xl, y)] = t2[i];
    }
  }
  __syncthreads();
}

// 1-D transforms of every row / column of the tile
template <int N, int CL, bool INV>
__device__ __forceinline__ void row_fft(float2 *slab, const float2 *tw) {
  fft_all<N, INV, AdjCfg<N, CL>::NT, AdjCfg<N, CL>::HR, true, RowB<N, CL>>(slab, tw);
}
template <int N, int CL, bool INV>
__device__ __forceinline__ void col_fft(float2 *slab, const float2 *tw) {
  fft_all<N, INV, AdjCfg<N, CL>::NT, AdjCfg<N, CL>::WC, false, ColA<N, CL>>(slab, tw);
}

struct AdjArgs {
  const float2 *O;
  int W;
  const void *frames;
  const int32_t *pos;
  const float *shift;     // n x 2 or nullptr
  const float2 *FP;       // F P, N x N
  const float2 *twiddle;  // N entries exp(-2 pi i m/N)
  float2 *gO;             // H x W (accumulated)
  float2 *gFP;            // N x N (accumulated)
  double *part;           // [n][CL][3]: loss, dL/d(dy), dL/d(dx)
  int frame0;             // first frame of this launch
};

template <int N, int CL, typename IT>
__global__ void __launch_bounds__(AdjCfg<N, CL>::NT, 1) amp_grad_kernel(AdjArgs a) {
  using C = AdjCfg<N, CL>;
  constexpr int WC = C::WC, HR = C::HR, NT = C::NT, E = C::E, NW = C::NW;
  constexpr float invK = 1.0f / (static_cast<float>(N) * static_cast<float>(N));
  extern __shared__ __align__(128) unsigned char smem[];
  float2 *slab = reinterpret_cast<float2 *>(smem);
  float2 *tw = reinterpret_cast<float2 *>(smem + C::OFF_TW);
  float2 *ps = reinterpret_cast<float2 *>(smem + C::OFF_AUX);
  double *red = reinterpret_cast<double *>(smem + C::OFF_RED);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int crank = 0;
  if constexpr (CL > 1) crank = static_cast<int>(cg::this_cluster().block_rank());
  const int f = a.frame0 + static_cast<int>(blockIdx.x) / CL;
  const int py = a.pos[2 * f], px = a.pos[2 * f + 1];
  const float dy = a.shift ? a.shift[2 * f] : 0.f, dx = a.shift ? a.shift[2 * f + 1] : 0.f;
  const IT *I = static_cast<const IT *>(a.frames) + static_cast<size_t>(f) * N * N;
  for (int m = tid; m < N; m += NT) tw[m] = a.twiddle[m];

  // 1. Z = FP . ph on column blocks, inverse transform -> Ps on row blocks
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int idx = tid + i * NT, y = idx / WC, xl = idx % WC, x = crank * WC + xl;
    slab[ColA<N, CL>::at(xl, y)] = cmul(a.FP[y * N + x], shift_phase<N>(y, x, dy, dx));
  }
  __syncthreads();
  col_fft<N, CL, true>(slab, tw);
  cols_to_rows<N, CL>(slab);
  row_fft<N, CL, true>(slab, tw);

  // 2. psi = Ps . O_j on row blocks (Ps kept), forward transform -> columns
  const float2 *Orow = a.O + static_cast<size_t>(py + crank * HR) * a.W + px;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int idx = tid + i * NT, yl = idx / N, x = idx % N;
    const float2 p = cscale(slab[RowB<N, CL>::at(yl, x)], invK);
    ps[yl * N + x] = p;
    slab[RowB<N, CL>::at(yl, x)] = cmul(p, Orow[static_cast<size_t>(yl) * a.W + x]);
  }
  __syncthreads();
  row_fft<N, CL, false>(slab, tw);
  rows_to_cols<N, CL>(slab);
  col_fft<N, CL, false>(slab, tw);

  // 3. G = 2 (|Psi| - sqrt I) Psi/|Psi| on columns; loss terms; F^H -> rows
  float loss = 0.f;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int idx = tid + i * NT, y = idx / WC, xl = idx % WC, x = crank * WC + xl;
    const float r = sqrtf(fmaxf(ival(I[y * N + x]), 0.f));
    const float2 v = slab[ColA<N, CL>::at(xl, y)];
    const float a2 = v.x * v.x + v.y * v.y;
    float2 g = make_float2(0.f, 0.f);
    float amp = 0.f;
    if (a2 > 0.f) {
      amp = sqrtf(a2);
      g = cscale(v, 2.f * (amp - r) / amp);
    }
    loss = fmaf(amp - r, amp - r, loss);
    slab[ColA<N, CL>::at(xl, y)] = g;
  }
  __syncthreads();
  col_fft<N, CL, true>(slab, tw);
  cols_to_rows<N, CL>(slab);
  row_fft<N, CL, true>(slab, tw);

  // 4. g_O += conj(Ps) g_psi; g_Ps = conj(O) g_psi, forward transform -> columns
  float2 *gOrow = a.gO + static_cast<size_t>(py + crank * HR) * a.W + px;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int idx = tid + i * NT, yl = idx / N, x = idx % N;
    const float2 gpsi = slab[RowB<N, CL>::at(yl, x)];
    const float2 p = ps[yl * N + x];
    const float2 go = cmulc(p, gpsi);
    float2 *dst = gOrow + static_cast<size_t>(yl) * a.W + x;
    atomicAdd(dst, go);  // one 8-byte vector reduction
    slab[RowB<N, CL>::at(yl, x)] = cmulc(Orow[static_cast<size_t>(yl) * a.W + x], gpsi);
  }
  __syncthreads();
  row_fft<N, CL, false>(slab, tw);
  rows_to_cols<N, CL>(slab);
  col_fft<N, CL, false>(slab, tw);

  // 5. position gradient and the probe-spectrum accumulation on columns
  float gdy = 0.f, gdx = 0.f;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int idx = tid + i * NT, y = idx / WC, xl = idx % WC, x = crank * WC + xl;
    const float2 gz = cscale(slab[ColA<N, CL>::at(xl, y)], invK);
    const float2 ph = shift_phase<N>(y, x, dy, dx);
    const float2 z = cmul(a.FP[y * N + x], ph);
    // Re(conj(gz) z (-2 pi i f / N)) = (2 pi f / N) Im(conj(gz) z)
    const float im = gz.x * z.y - gz.y * z.x;
    const float w = 2.0f * static_cast<float>(kPi) / static_cast<float>(N);
    gdy = fmaf(w * freq<N>(y), im, gdy);
    gdx = fmaf(w * freq<N>(x), im, gdx);
    const float2 acc = cmul(gz, make_float2(ph.x, -ph.y));
    atomicAdd(&a.gFP[y * N + x], acc);
  }
  const float s0 = warp_sum_f(loss), s1 = warp_sum_f(gdy), s2 = warp_sum_f(gdx);
  if (lane == 0) {
    red[warp] = s0;
    red[NW + warp] = s1;
    red[2 * NW + warp] = s2;
  }
  __syncthreads();
  if (tid == 0) {
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    for (int w = 0; w < NW; ++w) {
      t0 += red[w];
      t1 += red[NW + w];
      t2 += red[2 * NW + w];
    }
    double *o = a.part + (static_cast<size_t>(f) * CL + crank) * 3;
    o[0] = t0;
    o[1] = t1;
    o[2] = t2;
  }
  if constexpr (CL > 1) cg::this_cluster().sync();  // peers may still read this CTA's tile
}

// one 2-D transform of a single N x N array: out = scale * F(in) (or F^-1
// without 1/K when INV), in natural row-major order
template <int N, int CL, bool INV>
__global__ void __launch_bounds__(AdjCfg<N, CL>::NT, 1)
    fft2_single_kernel(const float2 *in, float2 *out, const float2 *twiddle, float scale) {
  using C = AdjCfg<N, CL>;
  constexpr int WC = C::WC, NT = C::NT, E = C::E;
  extern __shared__ __align__(128) unsigned char smem[];
  float2 *slab = reinterpret_cast<float2 *>(smem);
  float2 *tw = reinterpret_cast<float2 *>(smem + C::OFF_TW);
  int crank = 0;
  if constexpr (CL > 1) crank = static_cast<int>(cg::this_cluster().block_rank());
  for (int m = threadIdx.x; m < N; m += NT) tw[m] = twiddle[m];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int idx = threadIdx.x + i * NT, y = idx / WC, xl = idx % WC;
    slab[ColA<N, CL>::at(xl, y)] = in[y * N + crank * WC + xl];
  }
  __syncthreads();
  col_fft<N, CL, INV>(slab, tw);
  cols_to_rows<N, CL>(slab);
  row_fft<N, CL, INV>(slab, tw);
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int idx = threadIdx.x + i * NT, yl = idx / N, x = idx % N;
    out[(crank * C::HR + yl) * N + x] = cscale(slab[RowB<N, CL>::at(yl, x)], scale);
  }
  if constexpr (CL > 1) cg::this_cluster().sync();
}

// loss and position gradients from the per-CTA partials (fixed order)
__global__ void adj_finish_kernel(const double *part, int n, int cl, float *gshift, double *loss) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int f = threadIdx.x; f < n; f += 256) {
    double l = 0.0, gy = 0.0, gx = 0.0;
    for (int c = 0; c < cl; ++c) {
      const double *p = part + (static_cast<size_t>(f) * cl + c) * 3;
      l += p[0];
      gy += p[1];
      gx += p[2];
    }
    acc += l;
    if (gshift) {
      gshift[2 * f] = static_cast<float>(gy);
      gshift[2 * f + 1] = static_cast<float>(gx);
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = sh[0];
}

__global__ void twiddle_kernel(float2 *tw, int N) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < N) {
    float s, c;
    sincospif(-2.0f * static_cast<float>(m) / static_cast<float>(N), &s, &c);
    tw[m] = make_float2(c, s);
  }
}

template <class K>
cudaError_t launch_cluster(K kern, int grid, int cl, int nt, size_t smem, cudaStream_t st,
                           AdjArgs *args_adj, const float2 *in, float2 *out, const float2 *tw,
                           float scale) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid * cl, 1, 1);
  cfg.blockDim = dim3(nt, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (cl > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  if constexpr (std::is_same<K, void (*)(AdjArgs)>::value) {
    return cudaLaunchKernelEx(&cfg, kern, *args_adj);
  } else {
    return cudaLaunchKernelEx(&cfg, kern, in, out, tw, scale);
  }
}

template <int N, int CL, typename IT>
cudaError_t run_amp_grad(const epie_amp_grad_args *g, double *loss_host) {
  using C = AdjCfg<N, CL>;
  constexpr int K = N * N;
  cudaStream_t st = static_cast<cudaStream_t>(g->stream);
  unsigned char *base = static_cast<unsigned char *>(g->scratch);
  auto *FP = reinterpret_cast<float2 *>(base);
  auto *gFP = FP + K;
  auto *tw = gFP + K;
  auto *loss_d = reinterpret_cast<double *>(tw + 512);
  auto *part = loss_d + 2;
  cudaError_t e;
  twiddle_kernel<<<(N + 127) / 128, 128, 0, st>>>(tw, N);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(gFP, 0, sizeof(float2) * K, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(g->grad_object, 0,
                           sizeof(float2) * static_cast<size_t>(g->obj_h) * g->obj_w, st)) !=
      cudaSuccess)
    return e;
  // F P
  e = launch_cluster(fft2_single_kernel<N, CL, false>, 1, CL, C::NT, C::SMEM, st, nullptr,
                     reinterpret_cast<const float2 *>(g->probe), FP, tw, 1.0f);
  if (e != cudaSuccess) return e;
  AdjArgs a{};
  a.O = reinterpret_cast<const float2 *>(g->object);
  a.W = g->obj_w;
  a.frames = g->frames;
  a.pos = g->pos;
  a.shift = g->shift;
  a.FP = FP;
  a.twiddle = tw;
  a.gO = reinterpret_cast<float2 *>(g->grad_object);
  a.gFP = gFP;
  a.part = part;
  constexpr int kChunk = 4096;  // positions per launch
  for (int f0 = 0; f0 < g->n; f0 += kChunk) {
    a.frame0 = f0;
    const int m = g->n - f0 < kChunk ? g->n - f0 : kChunk;
    e = launch_cluster(amp_grad_kernel<N, CL, IT>, m, CL, C::NT, C::SMEM, st, &a, nullptr,
                       nullptr, nullptr, 0.f);
    if (e != cudaSuccess) return e;
  }
  // g_P = K F^-1(g_FP)
  e = launch_cluster(fft2_single_kernel<N, CL, true>, 1, CL, C::NT, C::SMEM, st, nullptr, gFP,
                     reinterpret_cast<float2 *>(g->grad_probe), tw, 1.0f);
  if (e != cudaSuccess) return e;
  adj_finish_kernel<<<1, 256, 0, st>>>(part, g->n, CL, g->grad_shift, loss_d);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (loss_host) {
    if ((e = cudaMemcpyAsync(loss_host, loss_d, sizeof(double), cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int N, int CL>
cudaError_t run_amp_grad_t(const epie_amp_grad_args *g, double *loss) {
  switch (g->intensity_dtype) {
    case EPIE_U16: return run_amp_grad<N, CL, uint16_t>(g, loss);
    case EPIE_F16: return run_amp_grad<N, CL, __half>(g, loss);
    default: return run_amp_grad<N, CL, float>(g, loss);
  }
}

int cl_for(int N) { return N == 64 ? 1 : (N == 128 ? 2 : 8); }

}  // namespace

extern "C" size_t epie_amp_grad_scratch_bytes(int32_t N, int32_t n) {
  if (!(N == 64 || N == 128 || N == 256) || n < 0) return 0;
  const size_t K = static_cast<size_t>(N) * N;
  return sizeof(float2) * (2 * K + 512) + sizeof(double) * (2 + 3 * static_cast<size_t>(n) * cl_for(N));
}

extern "C" int epie_amp_loss_grad(const epie_amp_grad_args *g, double *loss) {
  std::string &err = epie::init_error_sink();
  if (!g) {
    err = "epie_amp_loss_grad: args is NULL";
    return EPIE_EINVAL;
  }
  if (!(g->N == 64 || g->N == 128 || g->N == 256)) {
    err = "epie_amp_loss_grad: N must be 64, 128 or 256";
    return EPIE_EINVAL;
  }
  if (g->intensity_dtype < EPIE_U16 || g->intensity_dtype > EPIE_F32 || g->n < 1 ||
      g->obj_h < g->N || g->obj_w < g->N || !g->object || !g->probe || !g->frames || !g->pos ||
      !g->grad_object || !g->grad_probe || !g->scratch) {
    err = "epie_amp_loss_grad: bad arguments";
    return EPIE_EINVAL;
  }
  if (g->scratch_bytes < epie_amp_grad_scratch_bytes(g->N, g->n)) {
    err = "epie_amp_loss_grad: scratch smaller than epie_amp_grad_scratch_bytes(N, n)";
    return EPIE_EINVAL;
  }
  cudaError_t e;
  switch (g->N) {
    case 64: e = run_amp_grad_t<64, 1>(g, loss); break;
    case 128: e = run_amp_grad_t<128, 2>(g, loss); break;
    default: e = run_amp_grad_t<256, 8>(g, loss); break;
  }
  if (e != cudaSuccess) {
    err = std::string("epie_amp_loss_grad: ") + cudaGetErrorString(e);
    return EPIE_ECUDA;
  }
  return EPIE_OK;
}
