// epie_peak.cu -- FP32 FMA-chain throughput of the device, the denominator
// the fused step kernel is measured against (its transforms run on the FP32
// CUDA cores, not the tensor cores).
//
// Every thread runs 8 independent chains a <- a * b + c (one FFMA each, 2
// FLOP); enough warps per SM hide the FMA latency, so the rate is the FP32
// pipe's.  Thread 0 of block 0 samples clock64() and %globaltimer at both
// ends, which gives the SM clock the rate was measured at.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/epie.h"
#include "epie_fft.cuh"

namespace epie {

namespace {

constexpr int PEAK_CHAINS = 8, PEAK_UNROLL = 32, PEAK_THREADS = 256;

__global__ void __launch_bounds__(PEAK_THREADS) fma_chain_kernel(int iters, float b, float c,
                                                                 float *sink, long long *clk) {
  long long c0 = 0;
  uint64_t t0 = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    t0 = global_ns();
    c0 = clock64();
  }
  float a[PEAK_CHAINS];
#pragma unroll
  for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = static_cast<float>(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
      for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < PEAK_CHAINS; ++k) s += a[k];
  if (s == 1234.5f) sink[threadIdx.x] = s;  // keeps the chains live; never true in practice
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    clk[0] = clock64() - c0;
    clk[1] = static_cast<long long>(global_ns() - t0);
  }
}

}  // namespace

int fma_peak(int device, int iters, double *tflops, double *sm_mhz, std::string *err) {
  int sms = 0;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  float *sink = nullptr;
  long long *clk = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float) * PEAK_THREADS);
  if (e == cudaSuccess) e = cudaMalloc(&clk, sizeof(long long) * 2);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int blocks = sms * 8;  // 64 warps per SM
  long long hclk[2] = {0, 0};
  float ms = 0.f;
  if (e == cudaSuccess) {
    fma_chain_kernel<<<blocks, PEAK_THREADS>>>(iters / 8 + 1, 1.0000001f, 1e-7f, sink, clk);  // warm-up
    cudaEventRecord(e0);
    fma_chain_kernel<<<blocks, PEAK_THREADS>>>(iters, 1.0000001f, 1e-7f, sink, clk);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
  }
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaMemcpy(hclk, clk, sizeof(hclk), cudaMemcpyDeviceToHost);
  if (sink) cudaFree(sink);
  if (clk) cudaFree(clk);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return EPIE_ECUDA;
  }
  const double flop = 2.0 * PEAK_CHAINS * PEAK_UNROLL * static_cast<double>(iters) *
                      static_cast<double>(blocks) * PEAK_THREADS;
  *tflops = flop / (static_cast<double>(ms) * 1e-3) / 1e12;
  *sm_mhz = hclk[1] > 0 ? static_cast<double>(hclk[0]) / static_cast<double>(hclk[1]) * 1e3 : 0.0;
  return EPIE_OK;
}

}  // namespace epie
