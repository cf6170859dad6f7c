// epie_internal.h -- declarations shared by the host scheduler (epie_abi.cpp)
// and the kernels (epie_fused_*.cu, epie_aux.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

// CTAs per frame (thread-block cluster size) of the fused kernel per frame
// side; every CTA holds N*N/CTAS complex values, 16 per thread.
#ifndef EPIE_CTAS_64
#define EPIE_CTAS_64 1
#endif
#ifndef EPIE_CTAS_128
#define EPIE_CTAS_128 4
#endif
#ifndef EPIE_CTAS_256
#define EPIE_CTAS_256 8
#endif
#ifndef EPIE_CTAS_512
#define EPIE_CTAS_512 16
#endif

namespace epie {

// Arguments of one group launch of the fused ePIE kernel (and of the plain
// path's per-group kernels).  All pointers are device pointers.
struct GroupArgs {
  float2 *O;                  // object, H x W, row-major
  int W;                      // object row pitch (elements)
  const float2 *P;            // probe at group start, N x N
  const void *frames;         // device frame set [capacity][N][N], FFT order
  const float *dark;          // N x N FFT order, or nullptr
  const int32_t *pos;         // [capacity][2] patch top-left (y, x)
  const int32_t *members;     // frame ids of this group
  int n_members;
  float2 *probe_part;         // [n_members][N][N] probe-update partials
  double *err_part;           // [capacity][err_stride] sum (|Psi|-sqrt I)^2
  double *isum_part;          // [capacity][err_stride] sum I
  int err_stride;             // partial slots per frame
  const unsigned long long *pmax2;  // bits of max|P|^2 (double) of this group
  unsigned long long *pmax2_clear;  // slot to zero for the next group's max
  const double *omax2_global; // max|O|^2 over the object, or nullptr (patch max)
  const float2 *twiddle;      // N entries exp(-2 pi i m / N)
  float alpha, beta;
  int *err_flag;              // device status word (bounded waits)
  float2 *accO;               // mini-batch: object-update accumulator (H x W) or nullptr
  int *cnt;                   // mini-batch: per-pixel count of covering patches
  // device group table (graph replay): when gstart is set, this launch runs
  // group `group` with members members[gstart[group] .. gstart[group+1]) and
  // the grid is sized for the largest group; surplus clusters exit at once
  const int32_t *gstart;
  int group;
  // 1 when the launch follows the probe reduction of the previous group of
  // the same sweep: that reduction waited for the previous step kernel, so
  // the object is final and may be read before this kernel's dependency wait
  int o_early;
  // the frames' measured amplitudes sqrt(max(I - dark, 0)) in FFT order and
  // their per-frame intensity sums, derived at append; when set, the step
  // kernel copies its amplitude tile instead of converting raw intensities
  const float *amp;
  const double *amp_isum;
  // limit of every bounded device wait (0: the default of 2 s), and the
  // failure injection of the timeout tests: when set, the first CTA of the
  // launch never issues its intensity-tile copy, so its wait expires
  unsigned long long wait_ns;
  int inject_skip_copy;
};

// error-flag bits written by kernels
enum : int { FLAG_TMA_TIMEOUT = 1, FLAG_TC_TIMEOUT = 2 };

// fused kernel: one group, dispatch on N, intensity type and tile shape (cl:
// CTAs per frame, 0 = the default for N)
cudaError_t launch_fused(int N, int itype, const GroupArgs &a, cudaStream_t st, int cl = 0);
// CTAs per frame of the fused kernel for this N and tile shape (error slots
// per frame); 0 when that shape is not built
int fused_ctas_per_frame(int N, int cl = 0);
// dynamic shared memory of the fused kernel (for diagnostics)
size_t fused_smem_bytes(int N, int itype);

// probe update after a group: P += scale * sum_m part[m]; writes bits of
// max|P|^2 (double) into *pmax2_next (must be zero on entry)
cudaError_t launch_probe_reduce(float2 *P, const float2 *part, int n_members, int N, float scale,
                                unsigned long long *pmax2_next, cudaStream_t st);
// the same with the member count of group `group` read from the device table;
// scale = 1/count when mean != 0, else 1
cudaError_t launch_probe_reduce_table(float2 *P, const float2 *part, const int32_t *gstart,
                                      int group, int mean, int N, unsigned long long *pmax2_next,
                                      cudaStream_t st);
// copy of 8 bytes on the device (graph-safe)
cudaError_t launch_copy_u64(const unsigned long long *src, unsigned long long *dst,
                            cudaStream_t st);
// max|P|^2 of the probe into *pmax2 (zeroed by the kernel's caller)
cudaError_t launch_probe_max(const float2 *P, int K, unsigned long long *pmax2, cudaStream_t st);
// max|O|^2 over the object into *out (double)
cudaError_t launch_object_max(const float2 *O, long long n, double *out, unsigned long long *tmp,
                              cudaStream_t st);
// sweep error: E = sum e / sum s over frames [0, n_frames), fixed order
// blocks: device scratch of 2 * ERR_BLOCKS doubles (per handle: concurrent
// sweeps of several handles must not share it)
constexpr int ERR_BLOCKS = 128;
cudaError_t launch_error_reduce(const double *err_part, const double *isum_part, int n_frames,
                                int stride, double *out, double *blocks, cudaStream_t st);
// live ingest: raw DC-centred frames -> device set in FFT order (ifftshift)
cudaError_t launch_ingest(const void *raw, void *dst, int n, int N, int esize, cudaStream_t st);
// out[i] = (1/k) sum_q src[q][i] (q in order) for n complex values; src is a
// device array of k device pointers; out may be one of the sources
cudaError_t launch_average(const float2 *const *src, int k, float2 *out, long long n,
                           cudaStream_t st);
// p[0..n) = v
cudaError_t launch_fill(float2 *p, long long n, float2 v, cudaStream_t st);
// dark field: DC-centred float -> FFT order
cudaError_t launch_dark_ingest(const float *raw, float *dst, int N, cudaStream_t st);
// amp[f] = sqrt(max(I_f - dark, 0)) (fp32) and isum[f] = sum of
// max(I_f - dark, 0) (FP64) for frames [f0, f0 + n) of the frame set, in the
// layout the step kernel of tile shape cl (CTAs per frame, 0 = the default)
// reads: FFT order, or the tile layouts of the 1-CTA 128^2, the 256^2 and the
// 512^2 kernels
cudaError_t launch_amp_ingest(const void *frames, int itype, const float *dark, float *amp,
                              double *isum, int f0, int n, int N, int cl, cudaStream_t st);
// the same at N = 128 in the tile layout of the 1-CTA 128^2 step kernel
cudaError_t launch_amp_ingest_128(const void *frames, int itype, const float *dark, float *amp,
                                  double *isum, int f0, int n, cudaStream_t st);
// the same at N = 256, in the tile layout of the 256^2 step kernel
cudaError_t launch_amp_ingest_256(const void *frames, int itype, const float *dark, float *amp,
                                  double *isum, int f0, int n, cudaStream_t st);
// the same at N = 512, in the tile layout of the 512^2 step kernel
cudaError_t launch_amp_ingest_512(const void *frames, int itype, const float *dark, float *amp,
                                  double *isum, int f0, int n, cudaStream_t st);

// plain unfused path pieces; the gather writes psi = P . O_j (fp32), or with
// hi set its bf16 split hi / lo (interleaved complex, lo may be null)
cudaError_t launch_plain_gather(const GroupArgs &a, int N, float2 *psi, double *omax2,
                                cudaStream_t st, void *hi = nullptr, void *lo = nullptr);
cudaError_t launch_plain_modulus(const GroupArgs &a, int N, int itype, float2 *Psi,
                                 cudaStream_t st);
cudaError_t launch_plain_update(const GroupArgs &a, int N, const float2 *psi1,
                                const double *omax2, cudaStream_t st);
int plain_err_stride(int N);

// mini-batch path: accumulate object deltas / counts, then apply
cudaError_t launch_mb_accumulate(const GroupArgs &a, int N, const float2 *psi1,
                                 const double *omax2, float2 *accO, int *cnt, cudaStream_t st);
cudaError_t launch_mb_apply(float2 *O, float2 *accO, int *cnt, long long n, float alpha,
                            cudaStream_t st);
// the same over the batch's patches only (cheaper while batch x N^2 is below
// the object size); members from `members` or, with gstart, from the group
// table; grid sized for n_members
cudaError_t launch_mb_apply_local(float2 *O, float2 *accO, int *cnt, int W, const int32_t *pos,
                                  const int32_t *members, int n_members, const int32_t *gstart,
                                  int group, int N, float alpha, cudaStream_t st);

// failure injection for the timeout tests: the next `count` tcgen05 GEMM
// calls skip the first operand copy on CTA 0 and bound their waits by wait_ns
void tc_gemm_inject(int count, long long wait_ns);

// tensor-core DFT path (epie_gemm.cu)
// D[M x Nn] = sum_t A_t B_t^T on the tensor cores (tcgen05, epie_tc_gemm.cu);
// bf16 operands K-major, fp32 D with row pitch ldd; terms 1 or 3 (split bf16)
int tc_gemm_bf16(const void *A0, const void *A1, const void *B0, const void *B1, float *D,
                 long long M, int Nn, int K, int ldd, int terms, int *err_flag, cudaStream_t st,
                 std::string *err);
// the same product of Nn = 2 fn columns, written for the next DFT pass: row
// R = f fn + y of the product (row y of frame f, interleaved complex values
// at columns 2 x + c) goes to row f fn + x, columns 2 y + c of hi (bf16 of the
// value) and lo (bf16 of the value minus hi; lo may be null), row pitch 2 fn;
// fn a multiple of 32 and M of fn
int tc_gemm_bf16_tsplit(const void *A0, const void *A1, const void *B0, const void *B1, void *hi,
                        void *lo, long long M, int fn, int K, int terms, int *err_flag,
                        cudaStream_t st, std::string *err);
// the same with fp32 operands read as tf32 (kind::tf32); K a multiple of 32
int tc_gemm_tf32(const float *A0, const float *A1, const float *B0, const float *B1, float *D,
                 long long M, int Nn, int K, int ldd, int terms, int *err_flag, cudaStream_t st,
                 std::string *err);

// FP32 FMA-chain throughput (epie_peak.cu)
int fma_peak(int device, int iters, double *tflops, double *sm_mhz, std::string *err);

struct GemmPath;
GemmPath *gemm_path_create(int N, int precision, cudaStream_t st, std::string *err);
void gemm_path_destroy(GemmPath *g);
int gemm_path_group(GemmPath *g, const GroupArgs &a, int itype, cudaStream_t st, std::string *err,
                    int64_t *kernels);

}  // namespace epie
