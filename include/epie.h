/*
 * epie.h -- C ABI of the GB300 live ePIE engine.
 *
 * The engine reconstructs an object O (H x W complex) and an illumination
 * (probe) P (N x N complex) from far-field diffraction frames with ePIE
 * (Maiden & Rodenburg 2009), the algorithm the paper runs (Sec. "ePIE
 * Implementation"), in the paper's live mode: frames are appended to a
 * growing, device-resident set while sweeps continue (Sec. "Extensions of the
 * ePIE implementation"; Sec. "Live ePIE": between iterations the processing
 * thread loads new data and pushes intermediate state to a display).  The
 * object and probe sizes and the pixel grid are fixed at initialisation from
 * the nominal scan (Sec. "Determine parameters").
 *
 * One ePIE step at scan position j (patch top-left R_j = (y_j, x_j)):
 *   psi   = P . O_j                     O_j = O[y_j : y_j+N, x_j : x_j+N]
 *   Psi   = F psi                       unnormalised 2-D DFT, exp(-2 pi i k.r/N)
 *   Psi'  = sqrt(I_j) Psi/|Psi|         (sqrt(I_j) where |Psi| = 0)
 *   psi'  = F^-1 Psi'                   includes 1/N^2
 *   Delta = psi' - psi
 *   O_j  += alpha conj(P)/max|P|^2 Delta
 *   P    += beta conj(O_j,old)/max|O_j,old|^2 Delta     (pre-step O_j and P)
 * A zero maximum turns its update off.  I_j = max(frame_j - dark, 0) (NaN
 * counts as below 0), with the
 * frame's zero frequency moved from the detector centre (N/2, N/2) to index 0.
 * Sweep modes (every sweep visits each frame present at its start once, in a
 * random order drawn from the handle's seed and the sweep index, as the
 * paper's engine shuffles per iteration):
 *   EPIE_SEQUENTIAL  one position at a time (classic ePIE);
 *   EPIE_COLOURED    positions are grouped into colour classes whose patches
 *                    do not overlap (greedy first-fit in append order,
 *                    optionally with a cap on the class size); a
 *                    class runs in parallel from the probe at class start and
 *                    the probe moves by the mean of its members' updates;
 *                    with one member per class this is EPIE_SEQUENTIAL;
 *   EPIE_MINIBATCH   consecutive batches of `batch` positions share the
 *                    batch-start O and P; object updates are divided by the
 *                    per-pixel number of covering patches, probe updates
 *                    averaged (the overlapping object updates accumulate with
 *                    float atomics, so results reproduce to rounding only).
 * The sweep error is E = sum_j sum_k (|Psi_j| - sqrt(I_j))^2 / sum_j sum_k I_j
 * (the paper defines none), accumulated in FP64.
 *
 * Visiting order of sweep s: SplitMix64 stream with state
 * seed ^ (s * 0xD1B54A32D192ED03); Fisher-Yates (for i = n-1 .. 1,
 * j = next() mod (i+1)) over the frames (sequential, mini-batch) or over the
 * class ids and then, with the same stream, over each class's members listed
 * in append order (coloured).
 *
 * Conventions for every call:
 *   - Complex arrays are interleaved float32 (re, im), row-major.
 *   - Host buffers belong to the caller; a call has finished reading or
 *     writing them when it returns.  The engine owns all device memory.
 *   - Calls on one handle are serialised by a mutex; epie_iterate releases it
 *     between sweeps and, while another call waits for it, hands it over
 *     before the next sweep, so frames appended by another thread during
 *     epie_iterate join at the next sweep boundary (Sec. "Live ePIE").  An
 *     append waits on the device for the sweeps already queued, so it never
 *     overwrites frames they still read (after epie_truncate_frames).
 *   - Every call returns EPIE_OK (0) or a negative status; epie_error() then
 *     holds a message.  After EPIE_ECUDA or EPIE_ETIMEOUT the handle only
 *     accepts epie_error and epie_destroy (EPIE_ESTATE otherwise).
 *   - There is no CPU fallback: a host without a usable CUDA device gets
 *     EPIE_ECUDA from epie_init.
 */
#ifndef EPIE_H
#define EPIE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define EPIE_API __attribute__((visibility("default")))
#else
#define EPIE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct epie_ctx *epie_t;

/* status codes */
#define EPIE_OK 0
#define EPIE_EINVAL (-1)     /* bad argument, size or configuration            */
#define EPIE_ERANGE (-2)     /* a patch is not fully inside the object          */
#define EPIE_ECAPACITY (-3)  /* append beyond the capacity fixed at init        */
#define EPIE_ECUDA (-4)      /* CUDA error (device lost, out of memory, ...)    */
#define EPIE_ETIMEOUT (-5)   /* a bounded device-side wait expired              */
#define EPIE_ENUMERIC (-6)   /* the sweep error is not finite                   */
#define EPIE_ESTATE (-7)     /* handle unusable after a fatal error             */

/* intensity element types (as passed by the caller and as stored on device) */
#define EPIE_U16 0           /* uint16 counts                                    */
#define EPIE_F16 1           /* IEEE binary16                                    */
#define EPIE_F32 2           /* float32                                          */

/* sweep modes */
#define EPIE_SEQUENTIAL 0
#define EPIE_COLOURED 1
#define EPIE_MINIBATCH 2

/* normaliser of the probe update */
#define EPIE_OMAX_PATCH 0    /* max |O|^2 over the position's patch (default)    */
#define EPIE_OMAX_GLOBAL 1   /* max |O|^2 over the whole object at group start   */

/* compute path */
#define EPIE_PATH_FUSED 0    /* one fused kernel per group (default)            */
#define EPIE_PATH_PLAIN 1    /* separate gather / FFT / modulus / IFFT / update */
#define EPIE_PATH_GEMM 2     /* DFT as dense GEMMs on the tensor cores          */

/* operand precision of EPIE_PATH_GEMM (fp32 accumulation in every case) */
#define EPIE_GEMM_BF16 0     /* bf16 operands                                    */
#define EPIE_GEMM_TF32 1     /* tf32 operands                                    */
#define EPIE_GEMM_BF16X3 2   /* split bf16: hi*hi + hi*lo + lo*hi                */
#define EPIE_GEMM_FP32EMU 3  /* fp32 emulated on bf16 tensor cores (9 products)  */
#define EPIE_GEMM_TC_BF16 4  /* bf16 operands, this library's tcgen05 kernel     */
#define EPIE_GEMM_TC_BF16X3 5 /* split bf16, this library's tcgen05 kernel: the
                                three products share one TMEM accumulator       */
#define EPIE_GEMM_TC_TF32 6  /* operands rounded to nearest tf32, own tcgen05 kernel */
#define EPIE_GEMM_TC_TF32X3 7 /* split tf32 (x = hi + lo, hi = x with its low 13
                                mantissa bits cleared): hi*hi + hi*lo + lo*hi in
                                one TMEM accumulator, own tcgen05 kernel        */

/* flags */
#define EPIE_CHECKED 1u      /* keep O, P of the sweep start; restore them when
                                the sweep error is not finite                   */
#define EPIE_PROBE_SUM 2u    /* coloured: probe moves by the sum, not the mean  */
#define EPIE_FRAMES_FFT_ORDER 8u /* frames and dark field arrive in FFT order (zero
                                frequency at [0,0]) and are stored as given;
                                without it they are DC-centred (the detector's
                                layout) and re-laid out on the device         */
#define EPIE_RAW_INTENSITY 16u /* fused path: the step kernel copies the stored
                                intensity rows (uint16 / FP16 / FP32) by TMA
                                and forms sqrt(max(I - dark, 0)) itself,
                                instead of reading amplitudes derived at append
                                (half the bytes per frame for uint16 and FP16,
                                no amplitude buffer of capacity x N^2 floats) */
#define EPIE_GRAPH 4u        /* fused path: capture a sweep's launches in a CUDA
                                graph once and replay it each sweep (the group
                                table is uploaded per sweep; recaptured when the
                                frame set or the dark field changes)           */

typedef struct {
  int32_t N;               /* frame side: 64, 128, 256 or 512 (2^n frames, Sec.
                              "ePIE Implementation")                            */
  int32_t obj_h, obj_w;    /* object size, fixed at init (Sec. "Determine
                              parameters"); each >= N                           */
  int32_t capacity;        /* maximum number of frames ever held on device     */
  int32_t intensity_dtype; /* EPIE_U16 | EPIE_F16 | EPIE_F32                    */
  int32_t mode;            /* EPIE_SEQUENTIAL | EPIE_COLOURED | EPIE_MINIBATCH  */
  int32_t batch;           /* EPIE_MINIBATCH: positions per batch (>= 1)        */
  int32_t omax_mode;       /* EPIE_OMAX_PATCH | EPIE_OMAX_GLOBAL                */
  int32_t path;            /* EPIE_PATH_FUSED | EPIE_PATH_PLAIN | EPIE_PATH_GEMM */
  float alpha, beta;       /* update strengths; the paper uses 1 and 1          */
  uint64_t seed;           /* visiting-order seed                              */
  int32_t device;          /* CUDA device ordinal                              */
  void *stream;            /* cudaStream_t to run on, or NULL for an own stream */
  uint32_t flags;          /* EPIE_CHECKED | EPIE_PROBE_SUM                     */
  int32_t class_cap;       /* EPIE_COLOURED: at most this many frames per colour
                              class (first-fit skips full classes); 0 = no cap  */
  int32_t gemm_precision;  /* EPIE_PATH_GEMM: EPIE_GEMM_*                        */
  int32_t ctas_per_frame;  /* EPIE_PATH_FUSED, the step kernel's tile shape: CTAs
                              (one cluster) per frame; 0 = the default (1, 4, 8,
                              16 for N = 64, 128, 256, 512); N = 128 also builds
                              1 and 2 (see the autotuner)                       */
} epie_config;

/* Fills *cfg with defaults: N 256, object 1024^2, capacity 1024, EPIE_U16,
 * EPIE_COLOURED, batch 64, EPIE_OMAX_PATCH, EPIE_PATH_FUSED, alpha = beta = 1,
 * seed 0, device 0, own stream, no flags, no class cap, EPIE_GEMM_BF16X3,
 * the default tile shape. */
EPIE_API void epie_config_default(epie_config *cfg);

/* Creates a handle and allocates every device buffer the configuration needs:
 * on the fused path that includes capacity*N*N fp32 measured amplitudes
 * beside the capacity*N*N frames of intensity_dtype.
 * probe0: N*N complex (required).  object0: obj_h*obj_w complex, or NULL for
 * an object of ones (the paper's "identity" start, Sec. "Results").
 * Returns EPIE_EINVAL for a bad configuration, EPIE_ECUDA when the device
 * cannot be used or memory runs out (*out is then NULL). */
EPIE_API int epie_init(epie_t *out, const epie_config *cfg, const float *probe0, const float *object0);

/* Dark-offset field subtracted from every frame (clamped at 0) before the
 * modulus replacement.  dark: N*N float32 in the detector (DC-centred) layout
 * of the frames (FFT order with EPIE_FRAMES_FFT_ORDER), or NULL to remove it.
 * Takes effect at the next sweep.  On the fused path the frames' measured
 * amplitudes sqrt(max(I - dark, 0)) are derived at append and re-derived here
 * for every frame already appended (one pass over the frame set); the call
 * returns when that is done. */
EPIE_API int epie_set_dark(epie_t h, const float *dark);

/* Live ingest (paper, Sec. "Extensions of the ePIE implementation"): appends
 * n frames and their positions.  frames: n*N*N host values of the handle's
 * intensity type, DC-centred detector layout; pos_yx: n*(y, x) int32 patch
 * top-left object pixels.  The frames are copied (through pinned staging
 * unless `frames` is itself page-locked) and re-laid out on the device;
 * colour classes are extended.  Fails without side effects with
 * EPIE_ECAPACITY (would exceed capacity) or EPIE_ERANGE (a patch leaves the
 * object).  n = 0 is a no-op. */
EPIE_API int epie_append_frames(epie_t h, const void *frames, const int32_t *pos_yx, int32_t n);

/* As epie_append_frames, with `frames_dev` a device pointer (n*N*N values,
 * same layout) that must stay valid until the call returns. */
EPIE_API int epie_append_frames_device(epie_t h, const void *frames_dev, const int32_t *pos_yx,
                              int32_t n);

/* Drops every frame appended after the first n_keep (to re-attach to a
 * restarted scan, paper Sec. "Live processing"); colour classes revert to
 * their state at n_keep frames.  0 <= n_keep <= current count. */
EPIE_API int epie_truncate_frames(epie_t h, int32_t n_keep);

/* Runs n_sweeps sweeps (n_sweeps >= 0) over the frames present at the start
 * of each sweep.  err_per_sweep: n_sweeps doubles receiving the sweep error
 * E, or NULL.  Returns EPIE_ENUMERIC if a sweep error is not finite (with
 * EPIE_CHECKED, O and P are then back at that sweep's start).  A sweep over
 * zero frames leaves the state unchanged and reports E = 0. */
EPIE_API int epie_iterate(epie_t h, int32_t n_sweeps, double *err_per_sweep);

/* Several independent scans (handles, each with its own stream) sweep
 * concurrently: every sweep of every handle is enqueued before any is waited
 * for, so colour classes of different scans share the GPU.  err: k*n_sweeps
 * doubles (handle-major) or NULL.  Returns the first failing handle's status
 * (its message in epie_error(handle)); the other handles finish their sweeps. */
EPIE_API int epie_iterate_many(epie_t *handles, int32_t k, int32_t n_sweeps, double *err);

/* The paper's parallel scheme (Sec. "Simulating live and parallel
 * processing": disjoint subsets iterated independently, then object and
 * illumination averaged for synchronisation): replaces the object and probe
 * of every handle by their mean over the k handles (FP32, summed in handle
 * order).  All handles must share N, the object size and the device. */
EPIE_API int epie_average_state(epie_t *handles, int32_t k);

/* Object (obj_h*obj_w complex) and probe (N*N complex) export / import at a
 * sweep boundary (paper, Sec. "Discussion": import and export of object and
 * illumination through the API).  n_floats must equal 2*obj_h*obj_w or
 * 2*N*N. */
EPIE_API int epie_get_object(epie_t h, float *dst, size_t n_floats);
EPIE_API int epie_get_probe(epie_t h, float *dst, size_t n_floats);
EPIE_API int epie_set_object(epie_t h, const float *src, size_t n_floats);
EPIE_API int epie_set_probe(epie_t h, const float *src, size_t n_floats);

/* Number of frames held; number of colour classes. */
EPIE_API int epie_num_frames(epie_t h, int32_t *n);
EPIE_API int epie_num_classes(epie_t h, int32_t *n);

/* Colour class of each of the first n frames (n <= frame count). */
EPIE_API int epie_get_colours(epie_t h, int32_t *colour, int32_t n);

/* Visiting order of sweep `sweep` over the current frames, as the next
 * epie_iterate would run it: order[count] frame ids and group_start[n_groups+1]
 * offsets (a group shares the probe at group start).  order must hold the frame
 * count, group_start the frame count + 1. */
EPIE_API int epie_get_order(epie_t h, int64_t sweep, int32_t *order, int32_t *group_start,
                   int32_t *n_groups);

/* Index of the next sweep (starts at 0; used to draw its order).  Setting it
 * resumes a run that was exported and re-imported. */
EPIE_API int epie_get_sweep_index(epie_t h, int64_t *sweep);
EPIE_API int epie_set_sweep_index(epie_t h, int64_t sweep);

/* Frame count of each sweep of the most recent epie_iterate call on this
 * handle: the size of the frame set the sweep snapshotted when it started
 * (paper, Sec. "Live ePIE": frames appended by another thread join at the
 * next sweep).  *n_out receives the number of sweeps that call ran; the
 * first min(*n_out, cap) counts go to `counts` (host).  Callable while
 * another thread iterates (it takes the handle's mutex between sweeps).
 * EPIE_EINVAL for a NULL handle or output. */
EPIE_API int epie_last_sweep_frames(epie_t h, int32_t *counts, int32_t cap, int32_t *n_out);

/* Device time of the last epie_iterate call in milliseconds (CUDA events on
 * the handle's stream) and the number of kernels it launched. */
EPIE_API int epie_last_timing(epie_t h, double *ms, int64_t *kernels);

/* Failure injection for the tests of the bounded device waits.  No GPU
 * fault is involved: a bulk copy that is never issued leaves its mbarrier
 * incomplete, the wait for it expires after wait_ns, the kernel sets its
 * status word, lets everything it did issue land, frees its tensor memory
 * and returns; the host turns the status into EPIE_ETIMEOUT.
 *   what = EPIE_INJECT_STEP_COPY: the next `count` launches of the fused
 *          step kernel of handle h (fused path, EPIE_GRAPH off) skip the
 *          intensity-tile copy on their first CTA; epie_iterate then
 *          returns EPIE_ETIMEOUT and the handle is unusable (EPIE_ESTATE);
 *   what = EPIE_INJECT_TC_COPY: the next `count` calls of the tcgen05 GEMM
 *          (epie_tc_gemm_bf16 / _tf32, or the GEMM path) skip the first
 *          operand copy on CTA 0 and set FLAG bit 2 of their status word
 *          (h may be NULL; process-wide).
 * wait_ns in [1e3, 2e9] bounds every wait of the injected launches (the
 * default limit is 2 s).  Returns EPIE_EINVAL for other arguments. */
#define EPIE_INJECT_STEP_COPY 1
#define EPIE_INJECT_TC_COPY 2
EPIE_API int epie_inject_fault(epie_t h, int32_t what, int32_t count, int64_t wait_ns);

/* Total number of kernels this handle has launched since epie_init (all
 * calls: ingest, step, reductions; library calls such as cuFFT excluded). */
EPIE_API int epie_launch_count(epie_t h, int64_t *total);

/* Step-kernel timing.  While on, epie_iterate brackets every launch of the
 * position-update step (the fused kernel, or the plain path's gather ... update
 * sequence) with CUDA events on the handle's stream and resolves them at the
 * end of each sweep.  epie_kernel_timing returns the totals since the last
 * call (launches, summed device milliseconds, frames processed) and resets
 * them. */
EPIE_API int epie_set_kernel_timing(epie_t h, int32_t on);
EPIE_API int epie_kernel_timing(epie_t h, int64_t *launches, double *ms, int64_t *frames);

/* One ePIE group update on caller-owned device buffers, allocating no device
 * memory.  The paper has no counterpart: this entry point serves callers that
 * cannot allocate device memory themselves or through the engine -- a
 * detector or acquisition framework that owns the GPU's memory and lends out
 * fixed buffers, or a live loop that must not take the device-wide
 * synchronisation of cudaMalloc / cudaFree.
 *
 * It runs the same step as epie_iterate does for one group (one colour
 * class): every member's exit wave, far field, modulus replacement, object
 * patch update with the probe at group start, then the probe update by the
 * mean (probe_mean != 0) or the sum of the members' probe updates.
 *   object   device, obj_h*obj_w complex float32 (updated in place)
 *   probe    device, N*N complex float32 (updated in place)
 *   frames   device, n_frames*N*N intensities of type intensity_dtype in FFT
 *            order (zero frequency at index [0,0], not DC-centred)
 *   pos      device, n_frames*(y, x) int32 patch top-left positions
 *   members  device, n_members frame ids of the group; their patches must be
 *            pairwise disjoint when n_members > 1
 *   dark     device, N*N float32 in FFT order, or NULL
 *   err_terms host, 2 doubles receiving sum (|Psi| - sqrt I)^2 and sum I over
 *            the group, or NULL
 *   stream   cudaStream_t (NULL: the legacy default stream)
 * Alignment: frames and probe 16-byte aligned, object 8-byte, pos, members
 * and dark 4-byte; a misaligned pointer gives EPIE_EINVAL before any launch.
 * Every call synchronises `stream` twice: once to read the device-side
 * validation of members and positions before the step, and once at the end
 * to read the step kernel's status word, so an expired bounded wait always
 * returns EPIE_ETIMEOUT (err_terms given or not).
 * All scratch lives in one file-scope device array of about 36 MiB that every
 * GPU loading the library holds until exit; calls share it and it keeps the
 * last call's contents, so calls that overlap on the GPU (other streams,
 * other host threads) race.  Limits (scratch size): n_frames <= 16384,
 * n_members <= 1024, 256, 64, 16 for N = 64, 128, 256, 512; beyond them the
 * call returns EPIE_EINVAL without launching anything.  Member ids,
 * positions and disjointness are checked on the device before the step
 * (EPIE_EINVAL / EPIE_ERANGE).  The first call on a device looks the array's
 * device address up, uploads the twiddle tables and waits for the device to
 * finish that upload.
 * On failure epie_error(NULL) holds the reason. */
EPIE_API int epie_group_step_static(int32_t N, int32_t intensity_dtype, float *object,
                                    int32_t obj_h, int32_t obj_w, float *probe,
                                    const void *frames, int32_t n_frames, const int32_t *pos,
                                    const int32_t *members, int32_t n_members,
                                    const float *dark, float alpha, float beta,
                                    int32_t probe_mean, double *err_terms, void *stream);

/* Differentiable reconstruction: the amplitude loss
 *   L = sum_j sum_k ( |F(S_dj P . O_j)|(k) - sqrt(I_j(k)) )^2
 * over positions j with patch O_j = O[y_j : y_j+N, x_j : x_j+N] and the probe
 * shifted by the sub-pixel offset d_j = (dy, dx) as a Fourier shift
 * S_d P = F^-1[ F P . exp(-2 pi i (ky dy + kx dx)/N) ] (frequencies in FFT
 * order, k >= N/2 standing for k - N), together with its gradients.  ePIE
 * (paper, Sec. "ePIE Implementation") projects onto the set this loss
 * measures the distance to.  Gradients use dL/dRe + i dL/dIm (PyTorch's
 * convention for real losses of complex tensors); where |Psi| = 0 the
 * amplitude's gradient is taken as 0.  All pointers are device pointers
 * except `loss` (host, may be NULL; when given the call waits for the result).
 * The object and probe-spectrum gradients accumulate with float atomics, so
 * their last bits may vary between runs; the loss and the position gradients
 * are reduced in a fixed order.  N is 64, 128 or 256. */
typedef struct {
  int32_t N, intensity_dtype;  /* frame side; EPIE_U16 | EPIE_F16 | EPIE_F32      */
  int32_t obj_h, obj_w, n;     /* object size, number of positions              */
  const float *object;         /* obj_h*obj_w complex                           */
  const float *probe;          /* N*N complex                                   */
  const void *frames;          /* n*N*N intensities, FFT order (zero frequency
                                  at [0,0], see epie_frames_to_fft_order)        */
  const int32_t *pos;          /* n*(y, x) patch top-left, inside the object    */
  const float *shift;          /* n*(dy, dx) sub-pixel offsets, or NULL (zero)   */
  float *grad_object;          /* obj_h*obj_w complex, overwritten              */
  float *grad_probe;           /* N*N complex, overwritten                      */
  float *grad_shift;           /* n*2, overwritten, or NULL                     */
  void *scratch;               /* device scratch of scratch_bytes               */
  size_t scratch_bytes;        /* >= epie_amp_grad_scratch_bytes(N, n)           */
  void *stream;                /* cudaStream_t                                  */
} epie_amp_grad_args;
EPIE_API size_t epie_amp_grad_scratch_bytes(int32_t N, int32_t n);
EPIE_API int epie_amp_loss_grad(const epie_amp_grad_args *args, double *loss);

/* Detector layout (zero frequency at the centre (N/2, N/2)) -> FFT order,
 * on the device: dst[f][ky][kx] = src[f][(ky+N/2)%N][(kx+N/2)%N] for n frames
 * of intensity_dtype elements (the re-layout epie_append_frames applies).
 * src and dst must not overlap. */
EPIE_API int epie_frames_to_fft_order(const void *src, void *dst, int32_t n, int32_t N,
                                      int32_t intensity_dtype, void *stream);

/* Tensor-core product, the building block of EPIE_GEMM_TC_*:
 *   D[M x Nn] = sum over t < terms of A_t[M x K] . B_t[Nn x K]^T
 * with terms = 1 (A0 B0) or 3 (A0 B0 + A0 B1 + A1 B0, the split-bf16 product
 * of x = x_hi + x_lo).  The paper (Sec. "ePIE Implementation") runs the
 * projection through a DFT; a row of N interleaved complex values times the
 * 2N x 2N real twiddle matrix is that row's DFT, which is how the GEMM path
 * uses this call.  A_t, B_t: bf16 (uint16 bit patterns), row-major, K
 * contiguous; D: fp32, row pitch ldd floats.  All pointers are device
 * pointers, 16-byte aligned; A1 and B1 may be NULL when terms = 1.
 * M % 128 == 0, Nn % 128 == 0, K % 64 == 0, ldd >= Nn, ldd % 4 == 0, else
 * EPIE_EINVAL.  `status` is a device int32 the kernel ORs 2 into when one of
 * its bounded waits (2 s) expires; D is then incomplete.  Asynchronous on
 * `stream`; allocates nothing.  On failure epie_error(NULL) holds the
 * reason. */
EPIE_API int epie_tc_gemm_bf16(const void *A0, const void *A1, const void *B0, const void *B1,
                               float *D, int64_t M, int32_t Nn, int32_t K, int32_t ldd,
                               int32_t terms, int32_t *status, void *stream);

/* The same product with fp32 operands that the tensor cores read as tf32
 * (tcgen05 kind::tf32: sign, exponent and the top 10 mantissa bits).  With
 * terms = 3 and each operand split as x = hi + lo, both tf32-exact, the sum
 * carries about 21 significant bits.  K % 32 == 0; otherwise as
 * epie_tc_gemm_bf16. */
EPIE_API int epie_tc_gemm_tf32(const float *A0, const float *A1, const float *B0,
                               const float *B1, float *D, int64_t M, int32_t Nn, int32_t K,
                               int32_t ldd, int32_t terms, int32_t *status, void *stream);

/* FP32 FMA throughput of `device`: a kernel of independent FMA chains on
 * every SM (8 blocks of 256 threads per SM, `iters` x 256 FMAs per thread,
 * about 35 ms per 1000 iters on a GB300) after one short warm-up launch.
 * *tflops = 2 x FMAs / elapsed time; *sm_mhz = the SM clock during the run
 * (clock64 over %globaltimer on one SM).  This is the measured roofline
 * denominator of the fused step, whose transforms run on the FP32 pipes;
 * the paper has no counterpart.  Synchronous; EPIE_EINVAL for iters < 1 or
 * NULL outputs. */
EPIE_API int epie_fp32_fma_peak(int32_t device, int32_t iters, double *tflops, double *sm_mhz);

/* Message of the handle's last error (or of the last failed epie_init in
 * this thread when h is NULL).  Valid until the next call on the handle. */
EPIE_API const char *epie_error(epie_t h);

/* Releases the handle and its device memory.  NULL is a no-op. */
EPIE_API int epie_destroy(epie_t h);

#ifdef __cplusplus
}
#endif

#endif /* EPIE_H */
