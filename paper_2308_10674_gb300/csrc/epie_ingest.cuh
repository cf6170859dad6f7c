// epie_ingest.cuh -- the loads of the amplitude derivation at append: 8
// consecutive stored intensities of a detector row per 16-byte vector load,
// and the assignment of a 32-row tile of a frame to the lanes of a block so
// that every warp instruction reads 8 rows x 64 contiguous bytes and writes
// shared memory without bank conflicts.
//
// The derivation itself (amp = sqrt(max(I - dark, 0)), and the sum of
// max(I - dark, 0) for the error metric's normalisation) is the measured
// modulus that the Fourier-magnitude replacement of ePIE imposes (Sec. "ePIE
// Implementation"), formed once per frame.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "epie_fft.cuh"

namespace epie {

// 8 consecutive stored intensities (16-byte aligned)
template <typename IT>
struct Raw8;

template <>
struct Raw8<uint16_t> {
  uint4 v;
  __device__ __forceinline__ void load(const uint16_t *p) {
    v = __ldcs(reinterpret_cast<const uint4 *>(p));
  }
  __device__ __forceinline__ float at(int i) const {
    const uint32_t w = i < 2 ? v.x : i < 4 ? v.y : i < 6 ? v.z : v.w;
    return static_cast<float>((i & 1) ? (w >> 16) : (w & 0xffffu));
  }
};

template <>
struct Raw8<__half> {
  uint4 v;
  __device__ __forceinline__ void load(const __half *p) {
    v = __ldcs(reinterpret_cast<const uint4 *>(p));
  }
  __device__ __forceinline__ float at(int i) const {
    const uint32_t w = i < 2 ? v.x : i < 4 ? v.y : i < 6 ? v.z : v.w;
    const unsigned short b = static_cast<unsigned short>((i & 1) ? (w >> 16) : (w & 0xffffu));
    return __half2float(__ushort_as_half(b));
  }
};

template <>
struct Raw8<float> {
  float4 a, b;
  __device__ __forceinline__ void load(const float *p) {
    a = __ldcs(reinterpret_cast<const float4 *>(p));
    b = __ldcs(reinterpret_cast<const float4 *>(p) + 1);
  }
  __device__ __forceinline__ float at(int i) const {
    const float4 &q = i < 4 ? a : b;
    const int k = i & 3;
    return k == 0 ? q.x : k == 1 ? q.y : k == 2 ? q.z : q.w;
  }
};

// d[0..7] = dark[0..7] (32-byte aligned), or zeros without a dark field
__device__ __forceinline__ void dark8(const float *dark, float d[8]) {
  if (dark) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(dark));
    const float4 b = __ldg(reinterpret_cast<const float4 *>(dark) + 1);
    d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = a.w;
    d[4] = b.x; d[5] = b.y; d[6] = b.z; d[7] = b.w;
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) d[i] = 0.f;
  }
}

// v = max(I - dark, 0), NaN mapped to 0, as the step kernels' staged path
// forms it (a subtraction of 0 without a dark field leaves I unchanged)
__device__ __forceinline__ float clamp_sub(float I, float d) { return fmaxf(I - d, 0.f); }

// One lane's share of a 32-row tile of a frame with SN columns in a block of
// NT threads (NT / 32 warps, a multiple of 4).  Lane l of warp w takes tile
// row yl = 8 (w mod 4) + l / 4 and the 8-column chunks at
// c0 + (NT / 4) j, c0 = 32 (w / 4) + 8 (l mod 4), j = 0 .. J - 1: a warp
// instruction covers 8 rows x 32 columns, each row as 64 contiguous bytes of
// 16-bit values, and its shared-memory writes at row pitch SN + 1 fall in 32
// distinct banks.
template <int SN, int NT, typename IT>
struct TileLane {
  static constexpr int J = SN * 4 / NT;
  static_assert(NT % 128 == 0 && J >= 1 && J * NT == 4 * SN, "tile split");
  Raw8<IT> raw[J];
  int yl, c0;
  __device__ __forceinline__ TileLane()
      : yl(8 * ((threadIdx.x >> 5) & 3) + ((threadIdx.x & 31) >> 2)),
        c0(32 * (threadIdx.x >> 7) + 8 * (threadIdx.x & 3)) {}
  // the lane's chunks of detector row ky of frame fr (all loads in flight)
  __device__ __forceinline__ void load(const IT *fr, int ky) {
#pragma unroll
    for (int j = 0; j < J; ++j) raw[j].load(fr + static_cast<size_t>(ky) * SN + c0 + (NT / 4) * j);
  }
  // rows[yl * (SN + 1) + kx] = sqrt(max(I - dark, 0)) for the lane's chunks,
  // max(I - dark, 0) added into the two-sum (s, c)
  __device__ __forceinline__ void store(float *rows, const float *dark, int ky, float &s,
                                        float &c) const {
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int col = c0 + (NT / 4) * j;
      float d[8];
      dark8(dark ? dark + static_cast<size_t>(ky) * SN + col : nullptr, d);
      float *r = rows + yl * (SN + 1) + col;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float v = clamp_sub(raw[j].at(i), d[i]);
        two_sum_add(s, c, v);
        r[i] = sqrtf(v);
      }
    }
  }
};

}  // namespace epie
