// epie_static.cu -- epie_group_step_static: one ePIE group update on
// caller-owned device buffers that allocates no device memory.
//
// Some callers cannot allocate device memory: an acquisition or detector
// framework that owns the GPU's memory and lends out fixed buffers, a host
// process whose device memory is budgeted by another allocator, or a live
// loop that must not take the device-wide synchronisation a cudaMalloc or
// cudaFree implies.  For them this entry point keeps every scratch buffer the
// step needs (probe-update partials, error partials, the twiddle tables, the
// max|P|^2 slots, a status word) in one file-scope device array, so each GPU
// that loads the library holds kScratchBytes (about 36 MiB) until exit.
//
// The array's name is only a host-side stand-in for the device symbol: the
// host looks its device address up once per device (cudaGetSymbolAddress,
// with that device current) and passes that address to the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/epie.h"
#include "epie_internal.h"

namespace {

constexpr size_t kMiB = size_t(1) << 20;
constexpr size_t kPartBytes = 32 * kMiB;          // probe-update partials
constexpr int kMaxFrameIds = 16384;               // frame ids < this
constexpr int kMaxSlots = 16;                     // CTAs per frame of the fused kernel
constexpr size_t kErrBytes = sizeof(double) * kMaxFrameIds * kMaxSlots;
constexpr size_t kOffErr = kPartBytes;
constexpr size_t kOffIsum = kOffErr + kErrBytes;
constexpr size_t kOffTw = kOffIsum + kErrBytes;   // twiddles for 64, 128, 256, 512
constexpr size_t kTwBytes = sizeof(float2) * (64 + 128 + 256 + 512);
constexpr size_t kOffSmall = kOffTw + 8192;       // pmax[2], group error[2], status
constexpr size_t kScratchBytes = kOffSmall + 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceScratch {
  bool ready = false;
  unsigned char *base = nullptr;  // device address of g_scratch on this device
};
std::mutex g_mu;
DeviceScratch g_dev[64];

thread_local std::string *g_err_sink = nullptr;

size_t tw_offset(int N) {
  switch (N) {
    case 64: return 0;
    case 128: return sizeof(float2) * 64;
    case 256: return sizeof(float2) * (64 + 128);
    default: return sizeof(float2) * (64 + 128 + 256);
  }
}

// member ids in range, patches inside the object, patches of a group pairwise
// disjoint (bits 1, 2, 4 of *flag)
__global__ void validate_group_kernel(const int32_t *members, int n_members, const int32_t *pos,
                                      int n_frames, int N, int H, int W, int *flag) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  for (int m = t; m < n_members; m += nt) {
    const int f = members[m];
    if (f < 0 || f >= n_frames) {
      atomicOr(flag, 1);
      continue;
    }
    const int y = pos[2 * f], x = pos[2 * f + 1];
    if (y < 0 || x < 0 || y > H - N || x > W - N) atomicOr(flag, 2);
  }
  for (long long p = t; p < static_cast<long long>(n_members) * n_members; p += nt) {
    const int a = static_cast<int>(p / n_members), b = static_cast<int>(p % n_members);
    if (a >= b) continue;
    const int fa = members[a], fb = members[b];
    if (fa < 0 || fa >= n_frames || fb < 0 || fb >= n_frames) continue;
    if (abs(pos[2 * fa] - pos[2 * fb]) < N && abs(pos[2 * fa + 1] - pos[2 * fb + 1]) < N)
      atomicOr(flag, 4);
  }
}

// sum of the members' error partials in member order (one block)
__global__ void group_error_kernel(const double *e, const double *s, const int32_t *members,
                                   int n_members, int stride, double *out) {
  __shared__ double se[256], ss[256];
  double a = 0.0, b = 0.0;
  for (int m = threadIdx.x; m < n_members; m += 256)
    for (int c = 0; c < stride; ++c) {
      a += e[static_cast<size_t>(members[m]) * stride + c];
      b += s[static_cast<size_t>(members[m]) * stride + c];
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
    out[0] = se[0];
    out[1] = ss[0];
  }
}

int fail(int code, const std::string &msg) {
  if (g_err_sink) *g_err_sink = "epie_group_step_static: " + msg;
  return code;
}

// once per device, with that device current
int setup_device(int dev, unsigned char **base) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= 64) return fail(EPIE_EINVAL, "device ordinal out of range");
  DeviceScratch &d = g_dev[dev];
  if (!d.ready) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess)
      return fail(EPIE_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    d.base = static_cast<unsigned char *>(p);
    float2 tw[64 + 128 + 256 + 512];
    for (int N : {64, 128, 256, 512}) {
      float2 *t = tw + tw_offset(N) / sizeof(float2);
      for (int m = 0; m < N; ++m) {
        const double ang = -2.0 * 3.14159265358979323846 * m / N;
        t[m] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
      }
    }
    e = cudaMemcpy(d.base + kOffTw, tw, kTwBytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
      return fail(EPIE_ECUDA, std::string("twiddle upload: ") + cudaGetErrorString(e));
    // a copy from pageable memory may return before its DMA lands: wait for
    // it here, so that a first call on a non-blocking stream never reads the
    // tables early
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess)
      return fail(EPIE_ECUDA, std::string("twiddle upload: ") + cudaGetErrorString(e));
    d.ready = true;
  }
  *base = d.base;
  return EPIE_OK;
}

}  // namespace

// the thread's epie_error(NULL) message lives in epie_abi.cpp
namespace epie {
std::string &init_error_sink();
}

extern "C" int epie_group_step_static(int32_t N, int32_t intensity_dtype, float *object,
                                      int32_t obj_h, int32_t obj_w, float *probe,
                                      const void *frames, int32_t n_frames, const int32_t *pos,
                                      const int32_t *members, int32_t n_members,
                                      const float *dark, float alpha, float beta,
                                      int32_t probe_mean, double *err_terms, void *stream) {
  g_err_sink = &epie::init_error_sink();
  if (!(N == 64 || N == 128 || N == 256 || N == 512))
    return fail(EPIE_EINVAL, "N must be 64, 128, 256 or 512");
  if (intensity_dtype < EPIE_U16 || intensity_dtype > EPIE_F32)
    return fail(EPIE_EINVAL, "bad intensity_dtype");
  if (!object || !probe || !frames || !pos || !members)
    return fail(EPIE_EINVAL, "object, probe, frames, pos and members are required");
  if (obj_h < N || obj_w < N || static_cast<long long>(obj_h) * obj_w > (1LL << 31))
    return fail(EPIE_EINVAL, "object must be at least N x N and below 2^31 pixels");
  if (n_frames < 1 || n_frames > kMaxFrameIds)
    return fail(EPIE_EINVAL, "n_frames must be in [1, 16384] (static scratch limit)");
  const size_t part_per_member = sizeof(float2) * static_cast<size_t>(N) * N;
  const int max_members = static_cast<int>(kPartBytes / part_per_member);
  if (n_members < 1 || n_members > max_members)
    return fail(EPIE_EINVAL, "n_members must be in [1, " + std::to_string(max_members) +
                                 "] for N = " + std::to_string(N) + " (static scratch limit)");
  if (!std::isfinite(alpha) || !std::isfinite(beta))
    return fail(EPIE_EINVAL, "alpha and beta must be finite");
  // the step kernel copies frame rows with bulk copies (16-byte aligned
  // source), reads the object as float2 and the probe reduction reads and
  // writes the probe as float4
  auto misaligned = [](const void *p, uintptr_t a) {
    return (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0;
  };
  if (misaligned(frames, 16)) return fail(EPIE_EINVAL, "frames must be 16-byte aligned");
  if (misaligned(probe, 16)) return fail(EPIE_EINVAL, "probe must be 16-byte aligned");
  if (misaligned(object, 8)) return fail(EPIE_EINVAL, "object must be 8-byte aligned");
  if (misaligned(pos, 4) || misaligned(members, 4) || (dark && misaligned(dark, 4)))
    return fail(EPIE_EINVAL, "pos, members and dark must be 4-byte aligned");
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(EPIE_ECUDA, cudaGetErrorString(ce));
  unsigned char *base = nullptr;
  int rc = setup_device(dev, &base);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto *pmax = reinterpret_cast<unsigned long long *>(base + kOffSmall);
  auto *gerr = reinterpret_cast<double *>(base + kOffSmall + 16);
  auto *flag = reinterpret_cast<int *>(base + kOffSmall + 32);   // validation bits
  auto *kflag = reinterpret_cast<int *>(base + kOffSmall + 36);  // kernel status word
#define SK(expr)                                                                 \
  do {                                                                           \
    cudaError_t e_ = (expr);                                                     \
    if (e_ != cudaSuccess) return fail(EPIE_ECUDA, std::string(#expr ": ") + cudaGetErrorString(e_)); \
  } while (0)
  // the scratch keeps the previous call's contents: clear what starts at zero
  SK(cudaMemsetAsync(base + kOffSmall, 0, 64, st));
  validate_group_kernel<<<32, 256, 0, st>>>(members, n_members, pos, n_frames, N, obj_h, obj_w,
                                            flag);
  SK(cudaGetLastError());
  int hflag = 0;
  SK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  SK(cudaStreamSynchronize(st));
  if (hflag & 1) return fail(EPIE_EINVAL, "a member id is outside [0, n_frames)");
  if (hflag & 2) return fail(EPIE_ERANGE, "a member's patch is not inside the object");
  if (hflag & 4) return fail(EPIE_EINVAL, "patches of the group overlap");

  const int K = N * N;
  auto *P = reinterpret_cast<float2 *>(probe);
  SK(epie::launch_probe_max(P, K, pmax, st));
  epie::GroupArgs a{};
  a.O = reinterpret_cast<float2 *>(object);
  a.W = obj_w;
  a.P = P;
  a.frames = frames;
  a.dark = dark;
  a.pos = pos;
  a.members = members;
  a.n_members = n_members;
  a.probe_part = reinterpret_cast<float2 *>(base);
  a.err_part = reinterpret_cast<double *>(base + kOffErr);
  a.isum_part = reinterpret_cast<double *>(base + kOffIsum);
  a.err_stride = epie::fused_ctas_per_frame(N);
  a.pmax2 = pmax;
  a.pmax2_clear = pmax + 1;
  a.omax2_global = nullptr;
  a.twiddle = reinterpret_cast<const float2 *>(base + kOffTw + tw_offset(N));
  a.alpha = alpha;
  a.beta = beta;
  a.err_flag = kflag;
  a.accO = nullptr;
  a.cnt = nullptr;
  SK(epie::launch_fused(N, intensity_dtype, a, st));
  const float scale = probe_mean ? 1.0f / static_cast<float>(n_members) : 1.0f;
  SK(epie::launch_probe_reduce(P, a.probe_part, n_members, N, scale, pmax + 1, st));
  double h2[2] = {0.0, 0.0};
  if (err_terms) {
    group_error_kernel<<<1, 256, 0, st>>>(a.err_part, a.isum_part, members, n_members,
                                          a.err_stride, gerr);
    SK(cudaGetLastError());
    SK(cudaMemcpyAsync(h2, gerr, sizeof h2, cudaMemcpyDeviceToHost, st));
  }
  // the kernel status word is read back on every call, so an expired bounded
  // wait is always reported (the next call clears the word)
  SK(cudaMemcpyAsync(&hflag, kflag, sizeof(int), cudaMemcpyDeviceToHost, st));
  SK(cudaStreamSynchronize(st));
  if (hflag & epie::FLAG_TMA_TIMEOUT) return fail(EPIE_ETIMEOUT, "a bounded device wait expired");
  if (err_terms) {
    err_terms[0] = h2[0];
    err_terms[1] = h2[1];
  }
#undef SK
  return EPIE_OK;
}
