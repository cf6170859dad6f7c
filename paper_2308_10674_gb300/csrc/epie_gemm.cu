// epie_gemm.cu -- the ePIE step with the 2-D DFT done as dense GEMMs on the
// tensor cores (precision study).
//
// The paper's engine projects with a DFT on 2^n frames (Sec. "ePIE
// Implementation"); here the DFT of a group of G frames is four real GEMMs
// per direction-pair instead of an FFT.  A row of interleaved complex values
// (length N) times the real 2N x 2N matrix T with
//   T[2k][2j] = Re F_kj, T[2k+1][2j] = -Im F_kj, T[2k][2j+1] = Im F_kj,
//   T[2k+1][2j+1] = Re F_kj,       F_kj = exp(-+ 2 pi i k j / N)
// is the row's DFT, so all G*N rows transform in one [G N x 2N] x [2N x 2N]
// GEMM.  The column DFT is the same GEMM after a per-frame transpose:
//   gather psi -> rows -> transpose -> rows (spectrum, transposed) ->
//   modulus -> rows^-1 -> transpose -> rows^-1 -> update.
// The GEMMs are plain library GEMMs (cuBLAS); gather, transposes, precision
// splits, modulus and update are this engine's kernels.  Precisions:
//   EPIE_GEMM_BF16    bf16 operands, fp32 accumulation (one GEMM)
//   EPIE_GEMM_TF32    fp32 operands rounded to tf32 by the tensor cores
//   EPIE_GEMM_BF16X3  x = x_hi + x_lo in bf16; A B ~ Ah Bh + Ah Bl + Al Bh
//   EPIE_GEMM_FP32EMU cuBLAS' fp32 emulation on bf16 tensor cores
//   EPIE_GEMM_TC_BF16, EPIE_GEMM_TC_BF16X3: the bf16 and split-bf16 products
//     on this engine's own tcgen05 kernel (epie_tc_gemm.cu), the three
//     split products accumulated in one tensor-memory accumulator; here the
//     splits and the transposes are folded into the gather, the GEMM
//     epilogues and the modulus (tc_bf16_group)
//   EPIE_GEMM_TC_TF32, EPIE_GEMM_TC_TF32X3: the same kernel on fp32 operands
//     read as tf32 (kind::tf32); the plain form rounds its operands to the
//     nearest tf32 first, the split form takes hi = x with its low 13
//     mantissa bits cleared and lo = x - hi, both tf32-exact
// Twiddles are evaluated in double precision on the host (exact k j mod N).
#include <cublas_v2.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/epie.h"
#include "epie_fft.cuh"
#include "epie_internal.h"

namespace epie {

struct GemmPath {
  int N = 0, precision = 0, cap = 0;
  cublasHandle_t blas = nullptr;
  float *Tf = nullptr, *Ti = nullptr;                       // fp32 forward / inverse, 2N x 2N
  __nv_bfloat16 *Tf_hi = nullptr, *Tf_lo = nullptr, *Ti_hi = nullptr, *Ti_lo = nullptr;
  // transposed twiddles (K-major B operand of the tcgen05 kernel)
  __nv_bfloat16 *Tft_hi = nullptr, *Tft_lo = nullptr, *Tit_hi = nullptr, *Tit_lo = nullptr;
  // transposed twiddles split for the tf32 kernel (fp32 hi / lo)
  float *Tft32_hi = nullptr, *Tft32_lo = nullptr, *Tit32_hi = nullptr, *Tit32_lo = nullptr;
  float *F_hi = nullptr, *F_lo = nullptr;                   // tf32 split rows, cap * N * 2N
  float2 *psi = nullptr, *Y = nullptr;                      // cap * N * N complex each
  __nv_bfloat16 *D_hi = nullptr, *D_lo = nullptr;           // cap * N * 2N
  // own tcgen05 bf16 kernel: the transposed split products of the row passes
  __nv_bfloat16 *E_hi = nullptr, *E_lo = nullptr;           // cap * N * 2N
  double *omax = nullptr;                                   // cap
};

namespace {

__global__ void split_bf16_kernel(const float *__restrict__ x, __nv_bfloat16 *__restrict__ hi,
                                  __nv_bfloat16 *__restrict__ lo, long long n) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float v = x[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = h;
    if (lo) lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// out[b][j][i] = in[b][i][j] for G frames of N x N complex (32 x 32 tiles)
__global__ void transpose_frames_kernel(const float2 *__restrict__ in, float2 *__restrict__ out,
                                        int N) {
  __shared__ float2 t[32][33];
  const size_t base = static_cast<size_t>(blockIdx.z) * N * N;
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) t[r][threadIdx.x] = in[base + (by + r) * N + bx + threadIdx.x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8)
    out[base + (bx + r) * N + by + threadIdx.x] = t[threadIdx.x][r];
}

// modulus replacement on the transposed spectrum Xt[b][kx][ky] (1/N^2 folded
// in), or (hi set) its bf16 split written instead.  One block per 32 x 32
// tile (kx0, ky0) of a member: the intensities, stored [ky][kx], are read
// along kx into shared memory and used along ky, so both the frame and the
// spectrum are read in whole rows; error partials per tile (N^2 / 1024 per
// frame, the plain path's slots)
template <typename IT>
__global__ void tmodulus_kernel(GroupArgs a, int N, float2 *__restrict__ Xt,
                                __nv_bfloat162 *__restrict__ hi, __nv_bfloat162 *__restrict__ lo) {
  __shared__ float sI[32][33];
  __shared__ double se[8], ss[8];
  const int m = blockIdx.z, K = N * N, tx = threadIdx.x, ty = threadIdx.y;
  const int kx0 = 32 * blockIdx.x, ky0 = 32 * blockIdx.y;
  const int f = a.members[m];
  const IT *I = static_cast<const IT *>(a.frames) + static_cast<size_t>(f) * K;
  const float invK = 1.0f / (static_cast<float>(N) * static_cast<float>(N));
  float s = 0.f;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int ky = ky0 + ty + 8 * r, k = ky * N + kx0 + tx;
    float In = ival(I[k]);
    if (a.dark) In -= a.dark[k];
    In = fmaxf(In, 0.f);
    sI[ty + 8 * r][tx] = In;
  }
  __syncthreads();
  float e = 0.f;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int kx = kx0 + ty + 8 * r, ky = ky0 + tx;
    const size_t t = static_cast<size_t>(m) * K + static_cast<size_t>(kx) * N + ky;
    const float In = sI[tx][ty + 8 * r];
    const float sq = sqrtf(In);
    float2 v = Xt[t];
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
    if (hi) {
      // the split operand of the inverse transform, written in place of v
      const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
      hi[t] = h;
      if (lo) lo[t] = __floats2bfloat162_rn(v.x - __low2float(h), v.y - __high2float(h));
    } else {
      Xt[t] = v;
    }
    const float d = amp - sq;
    e = fmaf(d, d, e);
    s += In;
  }
  const int w = (ty * 32 + tx) >> 5;
  const float we = warp_sum_f(e), ws = warp_sum_f(s);
  if (tx == 0) {
    se[w] = we;
    ss[w] = ws;
  }
  __syncthreads();
  if (tx == 0 && ty == 0) {
    double te = 0.0, ts = 0.0;
    for (int q = 0; q < 8; ++q) {
      te += se[q];
      ts += ss[q];
    }
    const int slot = blockIdx.y * (N / 32) + blockIdx.x;
    a.err_part[static_cast<size_t>(f) * a.err_stride + slot] = te;
    a.isum_part[static_cast<size_t>(f) * a.err_stride + slot] = ts;
  }
}

// x = hi + lo with hi = x without its low 13 mantissa bits (tf32-exact) and
// lo = x - hi, exact in fp32 and itself tf32-exact
__global__ void split_tf32_kernel(const float *__restrict__ x, float *__restrict__ hi,
                                  float *__restrict__ lo, long long n) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float v = x[i];
    const float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
    hi[i] = h;
    lo[i] = v - h;
  }
}

// x rounded to the nearest tf32 value (ties to even; finite inputs)
__global__ void round_tf32_kernel(const float *__restrict__ x, float *__restrict__ r,
                                  long long n) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    uint32_t u = __float_as_uint(x[i]);
    u += 0xFFFu + ((u >> 13) & 1u);
    r[i] = __uint_as_float(u & 0xFFFFE000u);
  }
}

int grid_for(long long n, int nt, int cap) {
  long long g = (n + nt - 1) / nt;
  if (g > cap) g = cap;
  return g < 1 ? 1 : static_cast<int>(g);
}

cudaError_t split(const float *x, __nv_bfloat16 *hi, __nv_bfloat16 *lo, long long n,
                  cudaStream_t st) {
  split_bf16_kernel<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(x, hi, lo, n);
  return cudaGetLastError();
}

bool tc_bf16_precision(int p) { return p == EPIE_GEMM_TC_BF16 || p == EPIE_GEMM_TC_BF16X3; }
bool tc_tf32_precision(int p) { return p == EPIE_GEMM_TC_TF32 || p == EPIE_GEMM_TC_TF32X3; }
bool tc_precision(int p) { return tc_bf16_precision(p) || tc_tf32_precision(p); }
bool split_precision(int p) {
  return p == EPIE_GEMM_BF16 || p == EPIE_GEMM_BF16X3 || tc_bf16_precision(p);
}
bool x3_precision(int p) { return p == EPIE_GEMM_BF16X3 || p == EPIE_GEMM_TC_BF16X3; }

// nearest tf32 value (ties to even) of a finite fp32 value
float tf32_round(float v) {
  uint32_t u;
  std::memcpy(&u, &v, 4);
  u += 0xFFFu + ((u >> 13) & 1u);
  u &= 0xFFFFE000u;
  std::memcpy(&v, &u, 4);
  return v;
}

float tf32_hi(float v) {
  uint32_t u;
  std::memcpy(&u, &v, 4);
  u &= 0xFFFFE000u;
  std::memcpy(&v, &u, 4);
  return v;
}

// dst (rows x 2N fp32) = src (rows x 2N) * T, T the 2N x 2N twiddle matrix
int rows_dft(GemmPath *g, const float2 *src, float2 *dst, long long rows, bool inverse,
             int *err_flag, cudaStream_t st, std::string *err) {
  const int n2 = 2 * g->N;
  const float one = 1.f, zero = 0.f;
  const int M = static_cast<int>(rows);
  cublasStatus_t s = CUBLAS_STATUS_SUCCESS;
  const float *srcf = reinterpret_cast<const float *>(src);
  float *dstf = reinterpret_cast<float *>(dst);
  // the kernel takes rows in blocks of 128; the buffers hold an even number
  // of frames, so the rows past the group (N = 64, odd group) exist and
  // their results are never read
  const long long mrows = (rows + 127) / 128 * 128;
  if (g->precision == EPIE_GEMM_TC_TF32) {
    // operands rounded to nearest tf32 (the tensor cores would truncate)
    round_tf32_kernel<<<grid_for(rows * n2, 256, 152 * 16), 256, 0, st>>>(srcf, g->F_hi,
                                                                           rows * n2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      *err = cudaGetErrorString(e);
      return EPIE_ECUDA;
    }
    return tc_gemm_tf32(g->F_hi, nullptr, inverse ? g->Ti : g->Tf, nullptr, dstf, mrows, n2, n2,
                        n2, 1, err_flag, st, err);
  }
  if (g->precision == EPIE_GEMM_TC_TF32X3) {
    split_tf32_kernel<<<grid_for(rows * n2, 256, 152 * 16), 256, 0, st>>>(srcf, g->F_hi, g->F_lo,
                                                                           rows * n2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      *err = cudaGetErrorString(e);
      return EPIE_ECUDA;
    }
    return tc_gemm_tf32(g->F_hi, g->F_lo, inverse ? g->Tit32_hi : g->Tft32_hi,
                        inverse ? g->Tit32_lo : g->Tft32_lo, dstf, mrows, n2, n2, n2, 3, err_flag,
                        st, err);
  }
  if (g->precision == EPIE_GEMM_TF32 || g->precision == EPIE_GEMM_FP32EMU) {
    const cublasComputeType_t ct = g->precision == EPIE_GEMM_TF32
                                       ? CUBLAS_COMPUTE_32F_FAST_TF32
                                       : CUBLAS_COMPUTE_32F_EMULATED_16BFX9;
    s = cublasGemmEx(g->blas, CUBLAS_OP_N, CUBLAS_OP_N, n2, M, n2, &one, inverse ? g->Ti : g->Tf,
                     CUDA_R_32F, n2, srcf, CUDA_R_32F, n2, &zero, dstf, CUDA_R_32F, n2, ct,
                     CUBLAS_GEMM_DEFAULT);
  } else {
    const bool x3 = g->precision == EPIE_GEMM_BF16X3;
    cudaError_t e = split(srcf, g->D_hi, x3 ? g->D_lo : nullptr, rows * n2, st);
    if (e != cudaSuccess) {
      *err = cudaGetErrorString(e);
      return EPIE_ECUDA;
    }
    const __nv_bfloat16 *Th = inverse ? g->Ti_hi : g->Tf_hi, *Tl = inverse ? g->Ti_lo : g->Tf_lo;
    s = cublasGemmEx(g->blas, CUBLAS_OP_N, CUBLAS_OP_N, n2, M, n2, &one, Th, CUDA_R_16BF, n2,
                     g->D_hi, CUDA_R_16BF, n2, &zero, dstf, CUDA_R_32F, n2, CUBLAS_COMPUTE_32F,
                     CUBLAS_GEMM_DEFAULT);
    if (x3 && s == CUBLAS_STATUS_SUCCESS)
      s = cublasGemmEx(g->blas, CUBLAS_OP_N, CUBLAS_OP_N, n2, M, n2, &one, Th, CUDA_R_16BF, n2,
                       g->D_lo, CUDA_R_16BF, n2, &one, dstf, CUDA_R_32F, n2, CUBLAS_COMPUTE_32F,
                       CUBLAS_GEMM_DEFAULT);
    if (x3 && s == CUBLAS_STATUS_SUCCESS)
      s = cublasGemmEx(g->blas, CUBLAS_OP_N, CUBLAS_OP_N, n2, M, n2, &one, Tl, CUDA_R_16BF, n2,
                       g->D_hi, CUDA_R_16BF, n2, &one, dstf, CUDA_R_32F, n2, CUBLAS_COMPUTE_32F,
                       CUBLAS_GEMM_DEFAULT);
  }
  if (s != CUBLAS_STATUS_SUCCESS) {
    *err = "cublasGemmEx failed (status " + std::to_string(static_cast<int>(s)) + ")";
    return EPIE_ECUDA;
  }
  return EPIE_OK;
}

int transpose(GemmPath *g, const float2 *src, float2 *dst, int frames, cudaStream_t st,
              std::string *err) {
  dim3 grid(g->N / 32, g->N / 32, frames), block(32, 8);
  transpose_frames_kernel<<<grid, block, 0, st>>>(src, dst, g->N);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return EPIE_ECUDA;
  }
  return EPIE_OK;
}

}  // namespace

void gemm_path_destroy(GemmPath *g) {
  if (!g) return;
  if (g->blas) cublasDestroy(g->blas);
  void *ptrs[] = {g->Tf,     g->Ti,     g->Tf_hi,  g->Tf_lo, g->Ti_hi, g->Ti_lo,
                  g->Tft_hi, g->Tft_lo, g->Tit_hi, g->Tit_lo, g->psi,   g->Y,
                  g->D_hi,   g->D_lo,   g->omax,   g->Tft32_hi, g->Tft32_lo, g->Tit32_hi,
                  g->Tit32_lo, g->F_hi, g->F_lo, g->E_hi, g->E_lo};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete g;
}

GemmPath *gemm_path_create(int N, int precision, cudaStream_t st, std::string *err) {
  GemmPath *g = new GemmPath;
  g->N = N;
  g->precision = precision;
  if (cublasCreate(&g->blas) != CUBLAS_STATUS_SUCCESS || cublasSetStream(g->blas, st) != CUBLAS_STATUS_SUCCESS) {
    *err = "cuBLAS initialisation failed";
    gemm_path_destroy(g);
    return nullptr;
  }
  const int n2 = 2 * N;
  std::vector<float> Tf(static_cast<size_t>(n2) * n2), Ti(Tf.size());
  for (int k = 0; k < N; ++k)
    for (int j = 0; j < N; ++j) {
      const long m = (static_cast<long>(k) * j) % N;
      const double ang = -2.0 * 3.14159265358979323846 * static_cast<double>(m) / N;
      const float c = static_cast<float>(std::cos(ang)), s = static_cast<float>(std::sin(ang));
      // forward: F = c + i s; inverse (unnormalised): conj(F)
      Tf[(2 * k) * n2 + 2 * j] = c;      Tf[(2 * k + 1) * n2 + 2 * j] = -s;
      Tf[(2 * k) * n2 + 2 * j + 1] = s;  Tf[(2 * k + 1) * n2 + 2 * j + 1] = c;
      Ti[(2 * k) * n2 + 2 * j] = c;      Ti[(2 * k + 1) * n2 + 2 * j] = s;
      Ti[(2 * k) * n2 + 2 * j + 1] = -s; Ti[(2 * k + 1) * n2 + 2 * j + 1] = c;
    }
  const size_t tb = sizeof(float) * Tf.size(), hb = sizeof(__nv_bfloat16) * Tf.size();
  bool ok = cudaMalloc(&g->Tf, tb) == cudaSuccess && cudaMalloc(&g->Ti, tb) == cudaSuccess &&
            cudaMalloc(&g->Tf_hi, hb) == cudaSuccess && cudaMalloc(&g->Tf_lo, hb) == cudaSuccess &&
            cudaMalloc(&g->Ti_hi, hb) == cudaSuccess && cudaMalloc(&g->Ti_lo, hb) == cudaSuccess;
  ok = ok && cudaMemcpy(g->Tf, Tf.data(), tb, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(g->Ti, Ti.data(), tb, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && split(g->Tf, g->Tf_hi, g->Tf_lo, static_cast<long long>(Tf.size()), st) == cudaSuccess &&
       split(g->Ti, g->Ti_hi, g->Ti_lo, static_cast<long long>(Ti.size()), st) == cudaSuccess &&
       cudaStreamSynchronize(st) == cudaSuccess;
  if (ok && tc_precision(precision)) {
    // Tt[n][k] = T[k][n]: the twiddle matrix as a K-major B operand
    std::vector<float> Tft(Tf.size()), Tit(Ti.size());
    for (int k = 0; k < n2; ++k)
      for (int n = 0; n < n2; ++n) {
        Tft[static_cast<size_t>(n) * n2 + k] = Tf[static_cast<size_t>(k) * n2 + n];
        Tit[static_cast<size_t>(n) * n2 + k] = Ti[static_cast<size_t>(k) * n2 + n];
      }
    ok = cudaMalloc(&g->Tft_hi, hb) == cudaSuccess && cudaMalloc(&g->Tft_lo, hb) == cudaSuccess &&
         cudaMalloc(&g->Tit_hi, hb) == cudaSuccess && cudaMalloc(&g->Tit_lo, hb) == cudaSuccess;
    // the fp32 buffers are free again once the splits above have run
    ok = ok && cudaMemcpy(g->Tf, Tft.data(), tb, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(g->Ti, Tit.data(), tb, cudaMemcpyHostToDevice) == cudaSuccess &&
         split(g->Tf, g->Tft_hi, g->Tft_lo, static_cast<long long>(Tf.size()), st) == cudaSuccess &&
         split(g->Ti, g->Tit_hi, g->Tit_lo, static_cast<long long>(Ti.size()), st) == cudaSuccess &&
         cudaStreamSynchronize(st) == cudaSuccess;
    if (ok && precision == EPIE_GEMM_TC_TF32) {
      // the tensor cores keep the top 10 mantissa bits of an fp32 operand; give
      // them the twiddles already rounded to nearest tf32
      std::vector<float> fr(Tft.size()), ir(Tit.size());
      for (size_t i = 0; i < Tft.size(); ++i) {
        fr[i] = tf32_round(Tft[i]);
        ir[i] = tf32_round(Tit[i]);
      }
      ok = cudaMemcpy(g->Tf, fr.data(), tb, cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMemcpy(g->Ti, ir.data(), tb, cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (ok && precision == EPIE_GEMM_TC_TF32X3) {
      std::vector<float> fh(Tft.size()), fl(Tft.size()), ih(Tit.size()), il(Tit.size());
      for (size_t i = 0; i < Tft.size(); ++i) {
        fh[i] = tf32_hi(Tft[i]);
        fl[i] = Tft[i] - fh[i];
        ih[i] = tf32_hi(Tit[i]);
        il[i] = Tit[i] - ih[i];
      }
      ok = cudaMalloc(&g->Tft32_hi, tb) == cudaSuccess && cudaMalloc(&g->Tft32_lo, tb) == cudaSuccess &&
           cudaMalloc(&g->Tit32_hi, tb) == cudaSuccess && cudaMalloc(&g->Tit32_lo, tb) == cudaSuccess;
      ok = ok && cudaMemcpy(g->Tft32_hi, fh.data(), tb, cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMemcpy(g->Tft32_lo, fl.data(), tb, cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMemcpy(g->Tit32_hi, ih.data(), tb, cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMemcpy(g->Tit32_lo, il.data(), tb, cudaMemcpyHostToDevice) == cudaSuccess;
    }
  }
  if (!ok) {
    *err = "GEMM path: twiddle matrices could not be set up";
    gemm_path_destroy(g);
    return nullptr;
  }
  return g;
}

int gemm_path_reserve(GemmPath *g, int members, std::string *err) {
  if (members <= g->cap) return EPIE_OK;
  int cap = members > 2 * g->cap ? members : 2 * g->cap;
  cap += cap & 1;  // even: whole 128-row blocks at N = 64
  void *ptrs[] = {g->psi, g->Y, g->D_hi, g->D_lo, g->omax, g->F_hi, g->F_lo, g->E_hi, g->E_lo};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  g->psi = g->Y = nullptr;
  g->D_hi = g->D_lo = nullptr;
  g->E_hi = g->E_lo = nullptr;
  g->F_hi = g->F_lo = nullptr;
  g->omax = nullptr;
  g->cap = 0;
  const size_t K = static_cast<size_t>(g->N) * g->N;
  bool ok = cudaMalloc(&g->psi, sizeof(float2) * K * cap) == cudaSuccess &&
            cudaMalloc(&g->Y, sizeof(float2) * K * cap) == cudaSuccess &&
            cudaMalloc(&g->omax, sizeof(double) * cap) == cudaSuccess;
  if (ok && split_precision(g->precision)) {
    ok = cudaMalloc(&g->D_hi, sizeof(__nv_bfloat16) * 2 * K * cap) == cudaSuccess;
    if (ok && x3_precision(g->precision))
      ok = cudaMalloc(&g->D_lo, sizeof(__nv_bfloat16) * 2 * K * cap) == cudaSuccess;
  }
  if (ok && tc_bf16_precision(g->precision)) {
    ok = cudaMalloc(&g->E_hi, sizeof(__nv_bfloat16) * 2 * K * cap) == cudaSuccess;
    if (ok && x3_precision(g->precision))
      ok = cudaMalloc(&g->E_lo, sizeof(__nv_bfloat16) * 2 * K * cap) == cudaSuccess;
  }
  if (ok && tc_tf32_precision(g->precision))
    ok = cudaMalloc(&g->F_hi, sizeof(float) * 2 * K * cap) == cudaSuccess;
  if (ok && g->precision == EPIE_GEMM_TC_TF32X3)
    ok = cudaMalloc(&g->F_lo, sizeof(float) * 2 * K * cap) == cudaSuccess;
  if (!ok) {
    *err = "GEMM path: out of device memory for a group of " + std::to_string(cap);
    return EPIE_ECUDA;
  }
  g->cap = cap;
  return EPIE_OK;
}

namespace {

cudaError_t launch_tmodulus(const GroupArgs &a, int N, int itype, float2 *Xt, void *hi, void *lo,
                            cudaStream_t st) {
  dim3 grid(N / 32, N / 32, a.n_members), block(32, 8);
  auto *h = static_cast<__nv_bfloat162 *>(hi), *l = static_cast<__nv_bfloat162 *>(lo);
  if (itype == EPIE_U16) tmodulus_kernel<uint16_t><<<grid, block, 0, st>>>(a, N, Xt, h, l);
  else if (itype == EPIE_F16) tmodulus_kernel<__half><<<grid, block, 0, st>>>(a, N, Xt, h, l);
  else tmodulus_kernel<float><<<grid, block, 0, st>>>(a, N, Xt, h, l);
  return cudaGetLastError();
}

// The own tcgen05 kernel's bf16 forms, with the precision splits and the
// transposes folded into the producers: the gather writes the split exit
// wave; the row passes write their products transposed and split (the next
// pass's operand); the column pass writes fp32 and the modulus writes the
// split of its result:
//   gather -> D ; rows(D) -> E^T ; cols(E) -> Y ; modulus(Y) -> D ;
//   cols^-1(D) -> E^T ; rows^-1(E) -> psi' ; update.
// Every split is bf16(v), bf16(v - bf16(v)) as in split_bf16_kernel, so the
// result equals that of the unfolded sequence bit for bit.
int tc_bf16_group(GemmPath *g, const GroupArgs &a, int itype, cudaStream_t st, std::string *err,
                  int64_t *kernels) {
  const int N = g->N, G = a.n_members, n2 = 2 * N;
  const bool x3 = g->precision == EPIE_GEMM_TC_BF16X3;
  const int terms = x3 ? 3 : 1;
  const long long mrows = (static_cast<long long>(G) * N + 127) / 128 * 128;
  void *dlo = x3 ? g->D_lo : nullptr, *elo = x3 ? g->E_lo : nullptr;
  const void *tf_lo = x3 ? g->Tft_lo : nullptr, *ti_lo = x3 ? g->Tit_lo : nullptr;
  cudaError_t e = launch_plain_gather(a, N, g->psi, g->omax, st, g->D_hi, dlo);
  int rc = EPIE_OK;
  if (e == cudaSuccess) {
    if ((rc = tc_gemm_bf16_tsplit(g->D_hi, dlo, g->Tft_hi, tf_lo, g->E_hi, elo, mrows, N, n2,
                                  terms, a.err_flag, st, err)))  // along x
      return rc;
    if ((rc = tc_gemm_bf16(g->E_hi, elo, g->Tft_hi, tf_lo, reinterpret_cast<float *>(g->Y), mrows,
                           n2, n2, n2, terms, a.err_flag, st, err)))  // along y
      return rc;
    e = launch_tmodulus(a, N, itype, g->Y, g->D_hi, dlo, st);
  }
  if (e == cudaSuccess) {
    if ((rc = tc_gemm_bf16_tsplit(g->D_hi, dlo, g->Tit_hi, ti_lo, g->E_hi, elo, mrows, N, n2,
                                  terms, a.err_flag, st, err)))  // along y
      return rc;
    if ((rc = tc_gemm_bf16(g->E_hi, elo, g->Tit_hi, ti_lo, reinterpret_cast<float *>(g->psi),
                           mrows, n2, n2, n2, terms, a.err_flag, st, err)))  // along x
      return rc;
    e = a.accO ? launch_mb_accumulate(a, N, g->psi, g->omax, a.accO, a.cnt, st)
               : launch_plain_update(a, N, g->psi, g->omax, st);
  }
  if (e != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return EPIE_ECUDA;
  }
  // gather, modulus, update, 4 tcgen05 GEMMs
  *kernels += 7;
  return EPIE_OK;
}

}  // namespace

int gemm_path_group(GemmPath *g, const GroupArgs &a, int itype, cudaStream_t st,
                    std::string *err, int64_t *kernels) {
  const int N = g->N, G = a.n_members;
  int rc = gemm_path_reserve(g, G, err);
  if (rc) return rc;
  if (tc_bf16_precision(g->precision)) return tc_bf16_group(g, a, itype, st, err, kernels);
  const long long rows = static_cast<long long>(G) * N;
  cudaError_t e = launch_plain_gather(a, N, g->psi, g->omax, st);
  if (e != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return EPIE_ECUDA;
  }
  if ((rc = rows_dft(g, g->psi, g->Y, rows, false, a.err_flag, st, err))) return rc;   // along x
  if ((rc = transpose(g, g->Y, g->psi, G, st, err))) return rc;
  if ((rc = rows_dft(g, g->psi, g->Y, rows, false, a.err_flag, st, err))) return rc;   // along y
  if ((e = launch_tmodulus(a, N, itype, g->Y, nullptr, nullptr, st)) != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return EPIE_ECUDA;
  }
  if ((rc = rows_dft(g, g->Y, g->psi, rows, true, a.err_flag, st, err))) return rc;    // along y
  if ((rc = transpose(g, g->psi, g->Y, G, st, err))) return rc;
  if ((rc = rows_dft(g, g->Y, g->psi, rows, true, a.err_flag, st, err))) return rc;    // along x
  e = a.accO ? launch_mb_accumulate(a, N, g->psi, g->omax, a.accO, a.cnt, st)
             : launch_plain_update(a, N, g->psi, g->omax, st);
  if (e != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return EPIE_ECUDA;
  }
  // (the own kernel's bf16 forms took tc_bf16_group above)
  const bool split_launch = split_precision(g->precision) || tc_tf32_precision(g->precision);
  // gather, 2 transposes, modulus, update (+ 4 splits, + 4 tcgen05 GEMMs)
  *kernels += 5 + (split_launch ? 4 : 0) + (tc_precision(g->precision) ? 4 : 0);
  return EPIE_OK;
}

}  // namespace epie
