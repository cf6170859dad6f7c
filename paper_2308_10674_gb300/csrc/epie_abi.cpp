// epie_abi.cpp -- host side of the GB300 live ePIE engine: the C ABI of
// include/epie.h, device memory, the live frame set, colour classes, the
// per-sweep visiting order and the launch sequence of a sweep.
//
// The paper's engine (Sec. "ePIE Implementation") iterates over the
// diffraction patterns in a randomly shuffled order for a fixed number of
// iterations; its live extension (Sec. "Extensions of the ePIE
// implementation", Sec. "Live ePIE") adds patterns between iterations and
// exports intermediate object and illumination.  Here that control loop is
// native code around hand-written kernels; PyTorch is not involved.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cstdint>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/epie.h"
#include "epie_internal.h"

using epie::GroupArgs;

namespace {

thread_local std::string g_init_error;

// ------------------------------------------------------------------ order stream
// SplitMix64 (Steele, Lea & Flood 2014) with the sweep state of include/epie.h.
struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
};

void shuffle(int32_t *a, int32_t n, SplitMix64 &g) {
  for (int32_t i = n - 1; i >= 1; --i) {
    const int32_t j = static_cast<int32_t>(g.next() % static_cast<uint64_t>(i + 1));
    std::swap(a[i], a[j]);
  }
}

size_t esize_of(int dtype) { return dtype == EPIE_F32 ? 4 : 2; }

}  // namespace

namespace epie {
// the calling thread's epie_error(NULL) message
std::string &init_error_sink() { return g_init_error; }
}  // namespace epie

// ------------------------------------------------------------------ handle

struct epie_ctx {
  std::mutex mu;
  std::atomic<int> waiting{0};  // calls blocked on mu (epie_iterate yields to them)
  epie_config cfg{};
  std::string err;
  bool dead = false;
  int K = 0;                    // N*N
  long long HW = 0;             // obj_h*obj_w
  cudaStream_t st = nullptr;    // compute stream
  cudaStream_t up = nullptr;    // upload stream (appends)
  bool own_stream = false;
  cudaEvent_t ev_up = nullptr;  // last upload finished
  cudaEvent_t ev_st = nullptr;  // work queued on st so far (appends wait for it)
  cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;
  double last_ms = 0.0;
  int64_t last_kernels = 0;
  int64_t launches_total = 0;
  // step-kernel timing
  bool ktime = false;
  std::vector<cudaEvent_t> kev;   // pairs (start, stop)
  std::vector<int> kev_frames;
  int kev_used = 0;
  int64_t kt_launches = 0, kt_frames = 0;
  double kt_ms = 0.0;

  // device state
  float2 *O = nullptr, *P = nullptr, *twiddle = nullptr;
  void *frames = nullptr;
  int32_t *pos_d = nullptr, *order_d = nullptr;
  float *dark_d = nullptr;
  bool has_dark = false;
  // fused path: measured amplitudes sqrt(max(I - dark, 0)) of every frame in
  // FFT order (fp32) and their intensity sums (FP64), derived at append and
  // re-derived when the dark field changes
  float *amp = nullptr;
  double *amp_isum = nullptr;
  float2 *probe_part = nullptr;
  int part_cap = 0;             // members the probe_part buffer holds
  double *err_part = nullptr, *isum_part = nullptr;
  double *err_blocks = nullptr;         // 2 * ERR_BLOCKS block sums of the sweep error
  int err_stride = 1;
  unsigned long long *pmax2 = nullptr;  // [2] double bits
  int pslot = 0;                        // slot holding max|P|^2 of the current probe
  double *omax_glob = nullptr;
  unsigned long long *omax_tmp = nullptr;
  double *err_out = nullptr;            // per-sweep errors of one chunk
  int *flag_d = nullptr;
  // checked mode
  float2 *O_keep = nullptr, *P_keep = nullptr;
  // plain path
  float2 *psi = nullptr;
  int psi_cap = 0;
  double *omax_m = nullptr;
  std::map<int, cufftHandle> plans;
  // tensor-core DFT path
  epie::GemmPath *gemm = nullptr;
  // graph replay of a sweep (EPIE_GRAPH)
  int32_t *gstart_d = nullptr;          // device group table, capacity + 1
  int32_t *order_h[2] = {nullptr, nullptr}, *gstart_h[2] = {nullptr, nullptr};  // pinned
  cudaEvent_t ev_order[2] = {nullptr, nullptr};
  int order_buf = 0;
  double *err_sweep = nullptr;          // the graph's sweep error
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  long long gkey[6] = {-1, -1, -1, -1, -1, -1};
  // mini-batch accumulators
  float2 *accO = nullptr;
  int *cnt = nullptr;
  // staging for appends
  void *stage_h[2] = {nullptr, nullptr};
  void *stage_d = nullptr;
  size_t stage_bytes = 0;
  cudaEvent_t ev_stage[2] = {nullptr, nullptr};
  int stage_next = 0;
  double *err_h = nullptr;              // pinned copy of err_out

  // host state
  int32_t n_frames = 0;
  std::vector<int32_t> pos_h;           // 2 per frame
  std::vector<int32_t> colour;          // per frame
  std::vector<std::vector<int32_t>> classes;  // members in append order
  std::vector<std::vector<int32_t>> cells;    // frame ids per grid cell
  int cell_rows = 0, cell_cols = 0;
  std::vector<uint32_t> stamp;          // per class: last frame that marked it
  int64_t sweep = 0;
  std::vector<int32_t> iter_frames;     // frames of each sweep of the last epie_iterate
  // failure injection (epie_inject_fault): step launches still to inject, wait limit
  int inject_steps = 0;
  unsigned long long inject_wait_ns = 0;

  int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    if (code == EPIE_ECUDA || code == EPIE_ETIMEOUT) dead = true;
    return code;
  }
  int cuda_fail(cudaError_t e, const char *what) {
    return fail(EPIE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  }
};

#define CK(expr)                                     \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return h->cuda_fail(e_, #expr); \
  } while (0)

namespace {

// The handle's mutex for one call.  The caller is counted while it waits,
// so that a thread in epie_iterate lets it in at the next sweep boundary
// (a plain mutex would let the iterating thread re-take it at once).
class CallLock {
 public:
  explicit CallLock(epie_ctx *h) : h_(h) {
    h_->waiting.fetch_add(1);
    h_->mu.lock();
    h_->waiting.fetch_sub(1);
  }
  ~CallLock() { h_->mu.unlock(); }
  CallLock(const CallLock &) = delete;
  CallLock &operator=(const CallLock &) = delete;

 private:
  epie_ctx *h_;
};

int check_handle(epie_t h) {
  if (!h) return EPIE_EINVAL;
  if (h->dead) return h->fail(EPIE_ESTATE, "handle unusable after an earlier fatal error: %s",
                               h->err.c_str());
  return EPIE_OK;
}

// greedy first-fit colour of a new frame; frames conflict iff their patches
// overlap (|dy| < N and |dx| < N); classes holding class_cap frames are
// skipped.  A uniform grid of N x N cells finds the candidates.
void colour_append(epie_ctx *h, int32_t f) {
  const int N = h->cfg.N;
  const int y = h->pos_h[2 * f], x = h->pos_h[2 * f + 1];
  const int cy = y / N, cx = x / N;
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      const int ry = cy + dy, rx = cx + dx;
      if (ry < 0 || rx < 0 || ry >= h->cell_rows || rx >= h->cell_cols) continue;
      for (int32_t g : h->cells[static_cast<size_t>(ry) * h->cell_cols + rx]) {
        if (std::abs(h->pos_h[2 * g] - y) < N && std::abs(h->pos_h[2 * g + 1] - x) < N)
          h->stamp[h->colour[g]] = static_cast<uint32_t>(f) + 1u;
      }
    }
  int32_t c = 0;
  const int32_t nc = static_cast<int32_t>(h->classes.size());
  const size_t cap = h->cfg.class_cap > 0 ? static_cast<size_t>(h->cfg.class_cap) : SIZE_MAX;
  while (c < nc && (h->stamp[c] == static_cast<uint32_t>(f) + 1u || h->classes[c].size() >= cap))
    ++c;
  if (c == nc) {
    h->classes.emplace_back();
    h->stamp.push_back(0);
  }
  h->colour[f] = c;
  h->classes[c].push_back(f);
  h->cells[static_cast<size_t>(cy) * h->cell_cols + cx].push_back(f);
}

// visiting order of sweep s over the first n frames (include/epie.h)
void make_order(const epie_ctx *h, int64_t s, int32_t n, std::vector<int32_t> &order,
                std::vector<int32_t> &gstart) {
  SplitMix64 g{h->cfg.seed ^ (static_cast<uint64_t>(s) * 0xD1B54A32D192ED03ULL)};
  order.resize(n);
  gstart.clear();
  if (h->cfg.mode == EPIE_COLOURED) {
    const int32_t nc = static_cast<int32_t>(h->classes.size());
    std::vector<int32_t> cls(nc);
    for (int32_t c = 0; c < nc; ++c) cls[c] = c;
    shuffle(cls.data(), nc, g);
    int32_t p = 0;
    for (int32_t c : cls) {
      gstart.push_back(p);
      const int32_t a = p;
      for (int32_t f : h->classes[c])
        if (f < n) order[p++] = f;
      shuffle(order.data() + a, p - a, g);
    }
    gstart.push_back(p);
  } else {
    for (int32_t i = 0; i < n; ++i) order[i] = i;
    shuffle(order.data(), n, g);
    const int32_t B = h->cfg.mode == EPIE_MINIBATCH ? h->cfg.batch : 1;
    for (int32_t a = 0; a < n; a += B) gstart.push_back(a);
    gstart.push_back(n);
  }
}

int ensure_part(epie_ctx *h, int members) {
  if (members <= h->part_cap) return EPIE_OK;
  int cap = std::max(members, h->part_cap * 2);
  if (h->probe_part) cudaFree(h->probe_part);
  h->probe_part = nullptr;
  h->part_cap = 0;
  CK(cudaMalloc(&h->probe_part, sizeof(float2) * static_cast<size_t>(cap) * h->K));
  h->part_cap = cap;
  if (h->cfg.path == EPIE_PATH_PLAIN) {
    if (h->psi) cudaFree(h->psi);
    if (h->omax_m) cudaFree(h->omax_m);
    h->psi = nullptr;
    h->omax_m = nullptr;
    CK(cudaMalloc(&h->psi, sizeof(float2) * static_cast<size_t>(cap) * h->K));
    CK(cudaMalloc(&h->omax_m, sizeof(double) * cap));
    h->psi_cap = cap;
  }
  return EPIE_OK;
}

int get_plan(epie_ctx *h, int batch, cufftHandle *out) {
  auto it = h->plans.find(batch);
  if (it != h->plans.end()) {
    *out = it->second;
    return EPIE_OK;
  }
  cufftHandle p;
  int n[2] = {h->cfg.N, h->cfg.N};
  if (cufftPlanMany(&p, 2, n, nullptr, 1, h->K, nullptr, 1, h->K, CUFFT_C2C, batch) != CUFFT_SUCCESS)
    return h->fail(EPIE_ECUDA, "cufftPlanMany(batch %d) failed", batch);
  if (cufftSetStream(p, h->st) != CUFFT_SUCCESS) return h->fail(EPIE_ECUDA, "cufftSetStream failed");
  h->plans[batch] = p;
  *out = p;
  return EPIE_OK;
}

// One group: fused kernel (or the plain sequence), then the probe reduction.
int run_group(epie_ctx *h, const int32_t *members_d, int n_members, bool o_early,
              int64_t *kernels) {
  const int N = h->cfg.N;
  int rc = ensure_part(h, n_members);
  if (rc) return rc;
  const bool mb = h->cfg.mode == EPIE_MINIBATCH;
  GroupArgs a{};
  a.O = h->O;
  a.W = h->cfg.obj_w;
  a.P = h->P;
  a.frames = h->frames;
  a.dark = h->has_dark ? h->dark_d : nullptr;
  a.pos = h->pos_d;
  a.members = members_d;
  a.n_members = n_members;
  a.probe_part = h->probe_part;
  a.err_part = h->err_part;
  a.isum_part = h->isum_part;
  a.err_stride = h->err_stride;
  a.pmax2 = h->pmax2 + h->pslot;
  a.pmax2_clear = h->pmax2 + (h->pslot ^ 1);
  a.twiddle = h->twiddle;
  a.alpha = h->cfg.alpha;
  a.beta = h->cfg.beta;
  a.err_flag = h->flag_d;
  a.accO = mb ? h->accO : nullptr;
  a.cnt = mb ? h->cnt : nullptr;
  a.o_early = o_early && !h->ktime;  // timing events sit between the launches
  a.amp = h->amp;
  a.amp_isum = h->amp_isum;
  if (h->cfg.omax_mode == EPIE_OMAX_GLOBAL) {
    CK(epie::launch_object_max(h->O, h->HW, h->omax_glob, h->omax_tmp, h->st));
    a.omax2_global = h->omax_glob;
    *kernels += 2;
  }
  if (h->ktime) {
    if (h->kev_used + 2 > static_cast<int>(h->kev.size())) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        h->kev.push_back(e);
      }
      h->kev_frames.resize(h->kev.size() / 2);
    }
    h->kev_frames[h->kev_used / 2] = n_members;
    CK(cudaEventRecord(h->kev[h->kev_used], h->st));
  }
  if (h->cfg.path == EPIE_PATH_FUSED) {
    if (h->inject_steps > 0) {
      --h->inject_steps;
      a.inject_skip_copy = 1;
      a.wait_ns = h->inject_wait_ns;
    }
    CK(epie::launch_fused(N, h->cfg.intensity_dtype, a, h->st, h->cfg.ctas_per_frame));
    *kernels += 1;
  } else if (h->cfg.path == EPIE_PATH_GEMM) {
    std::string why;
    if ((rc = epie::gemm_path_group(h->gemm, a, h->cfg.intensity_dtype, h->st, &why, kernels)))
      return h->fail(rc, "GEMM path: %s", why.c_str());
  } else {
    cufftHandle plan;
    if ((rc = get_plan(h, n_members, &plan))) return rc;
    CK(epie::launch_plain_gather(a, N, h->psi, h->omax_m, h->st));
    auto *z = reinterpret_cast<cufftComplex *>(h->psi);
    if (cufftExecC2C(plan, z, z, CUFFT_FORWARD) != CUFFT_SUCCESS)
      return h->fail(EPIE_ECUDA, "cufftExecC2C forward failed");
    CK(epie::launch_plain_modulus(a, N, h->cfg.intensity_dtype, h->psi, h->st));
    if (cufftExecC2C(plan, z, z, CUFFT_INVERSE) != CUFFT_SUCCESS)
      return h->fail(EPIE_ECUDA, "cufftExecC2C inverse failed");
    if (mb)
      CK(epie::launch_mb_accumulate(a, N, h->psi, h->omax_m, h->accO, h->cnt, h->st));
    else
      CK(epie::launch_plain_update(a, N, h->psi, h->omax_m, h->st));
    *kernels += 3;  // gather, modulus, update (the two transforms are cuFFT's)
  }
  if (h->ktime) {
    CK(cudaEventRecord(h->kev[h->kev_used + 1], h->st));
    h->kev_used += 2;
  }
  if (mb) {
    // apply over the batch's patches while they cover less than the object
    if (static_cast<long long>(n_members) * h->K < h->HW)
      CK(epie::launch_mb_apply_local(h->O, h->accO, h->cnt, h->cfg.obj_w, h->pos_d, members_d,
                                     n_members, nullptr, 0, N, h->cfg.alpha, h->st));
    else
      CK(epie::launch_mb_apply(h->O, h->accO, h->cnt, h->HW, h->cfg.alpha, h->st));
    *kernels += 1;
  }
  const bool mean = h->cfg.mode == EPIE_MINIBATCH ||
                    (h->cfg.mode == EPIE_COLOURED && !(h->cfg.flags & EPIE_PROBE_SUM));
  const float scale = mean ? 1.0f / static_cast<float>(n_members) : 1.0f;
  CK(epie::launch_probe_reduce(h->P, h->probe_part, n_members, N, scale,
                               h->pmax2 + (h->pslot ^ 1), h->st));
  *kernels += 1;
  h->pslot ^= 1;
  return EPIE_OK;
}

int recompute_pmax(epie_ctx *h) {
  CK(cudaMemsetAsync(h->pmax2 + h->pslot, 0, sizeof(unsigned long long), h->st));
  CK(epie::launch_probe_max(h->P, h->K, h->pmax2 + h->pslot, h->st));
  h->launches_total += 1;
  return EPIE_OK;
}

// Graph replay of a fused-path sweep: the launches read their group from
// the device table, so one capture serves every sweep with the same number
// of groups and the same largest group.
int run_sweep_graph(epie_ctx *h, int slot, const std::vector<int32_t> &order,
                    const std::vector<int32_t> &gstart, int64_t *kernels) {
  const int32_t n = h->n_frames;
  const int ng = static_cast<int>(gstart.size()) - 1;
  int maxg = 0;
  for (int g = 0; g < ng; ++g) maxg = std::max(maxg, gstart[g + 1] - gstart[g]);
  int rc = ensure_part(h, maxg);
  if (rc) return rc;
  // upload the table through a pinned buffer that the previous use released
  const int b = h->order_buf;
  h->order_buf ^= 1;
  CK(cudaEventSynchronize(h->ev_order[b]));
  std::copy(order.begin(), order.end(), h->order_h[b]);
  std::copy(gstart.begin(), gstart.end(), h->gstart_h[b]);
  CK(cudaMemcpyAsync(h->order_d, h->order_h[b], sizeof(int32_t) * n, cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(h->gstart_d, h->gstart_h[b], sizeof(int32_t) * (ng + 1),
                     cudaMemcpyHostToDevice, h->st));
  CK(cudaEventRecord(h->ev_order[b], h->st));
  if (h->pslot != 0) {  // the captured sweep starts from slot 0
    CK(epie::launch_copy_u64(h->pmax2 + 1, h->pmax2, h->st));
    h->pslot = 0;
    *kernels += 1;
  }
  const long long key[6] = {n, ng, maxg, h->has_dark ? 1 : 0,
                            static_cast<long long>(reinterpret_cast<uintptr_t>(h->probe_part)),
                            h->cfg.omax_mode};
  if (!h->gexec || !std::equal(key, key + 6, h->gkey)) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
    {  // configure the kernel (shared-memory size, cluster shape) outside the capture
      GroupArgs z{};
      CK(epie::launch_fused(h->cfg.N, h->cfg.intensity_dtype, z, h->st, h->cfg.ctas_per_frame));
    }
    const int N = h->cfg.N;
    const bool mb = h->cfg.mode == EPIE_MINIBATCH;
    const int mean = mb || (h->cfg.mode == EPIE_COLOURED && !(h->cfg.flags & EPIE_PROBE_SUM));
    CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
    int p = 0;
    cudaError_t ce = cudaSuccess;
    for (int g = 0; g < ng && ce == cudaSuccess; ++g) {
      GroupArgs a{};
      a.O = h->O;
      a.W = h->cfg.obj_w;
      a.P = h->P;
      a.frames = h->frames;
      a.dark = h->has_dark ? h->dark_d : nullptr;
      a.pos = h->pos_d;
      a.members = h->order_d;
      a.n_members = maxg;  // grid size; the table gives the group's own size
      a.gstart = h->gstart_d;
      a.group = g;
      a.probe_part = h->probe_part;
      a.err_part = h->err_part;
      a.isum_part = h->isum_part;
      a.err_stride = h->err_stride;
      a.pmax2 = h->pmax2 + p;
      a.pmax2_clear = h->pmax2 + (p ^ 1);
      a.twiddle = h->twiddle;
      a.alpha = h->cfg.alpha;
      a.beta = h->cfg.beta;
      a.err_flag = h->flag_d;
      a.accO = mb ? h->accO : nullptr;
      a.cnt = mb ? h->cnt : nullptr;
      a.o_early = g > 0;
      a.amp = h->amp;
      a.amp_isum = h->amp_isum;
      if (h->cfg.omax_mode == EPIE_OMAX_GLOBAL) {
        ce = epie::launch_object_max(h->O, h->HW, h->omax_glob, h->omax_tmp, h->st);
        a.omax2_global = h->omax_glob;
      }
      if (ce == cudaSuccess)
        ce = epie::launch_fused(N, h->cfg.intensity_dtype, a, h->st, h->cfg.ctas_per_frame);
      if (ce == cudaSuccess && mb) {
        if (static_cast<long long>(maxg) * h->K < h->HW)
          ce = epie::launch_mb_apply_local(h->O, h->accO, h->cnt, h->cfg.obj_w, h->pos_d,
                                           h->order_d, maxg, h->gstart_d, g, N, h->cfg.alpha,
                                           h->st);
        else
          ce = epie::launch_mb_apply(h->O, h->accO, h->cnt, h->HW, h->cfg.alpha, h->st);
      }
      if (ce == cudaSuccess)
        ce = epie::launch_probe_reduce_table(h->P, h->probe_part, h->gstart_d, g, mean, N,
                                             h->pmax2 + (p ^ 1), h->st);
      p ^= 1;
    }
    if (ce == cudaSuccess && p == 1) ce = epie::launch_copy_u64(h->pmax2 + 1, h->pmax2, h->st);
    if (ce == cudaSuccess)
      ce = epie::launch_error_reduce(h->err_part, h->isum_part, n, h->err_stride, h->err_sweep,
                                     h->err_blocks, h->st);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(h->st, &graph);
    if (ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return h->cuda_fail(ce, "sweep capture");
    }
    if (ee != cudaSuccess) return h->cuda_fail(ee, "cudaStreamEndCapture");
    h->graph = graph;
    CK(cudaGraphInstantiate(&h->gexec, graph, 0));
    std::copy(key, key + 6, h->gkey);
  }
  CK(cudaGraphLaunch(h->gexec, h->st));
  CK(cudaMemcpyAsync(h->err_out + slot, h->err_sweep, sizeof(double), cudaMemcpyDeviceToDevice,
                     h->st));
  const bool mb = h->cfg.mode == EPIE_MINIBATCH;
  *kernels += static_cast<int64_t>(ng) * (2 + (mb ? 1 : 0) +
                                          (h->cfg.omax_mode == EPIE_OMAX_GLOBAL ? 2 : 0)) +
              2 + (ng % 2);
  return EPIE_OK;
}

// one sweep over the frames present now; writes the sweep error to err_out[slot]
int run_sweep(epie_ctx *h, int slot, int64_t *kernels) {
  const int32_t n = h->n_frames;
  CK(cudaStreamWaitEvent(h->st, h->ev_up, 0));
  if (h->cfg.flags & EPIE_CHECKED) {
    CK(cudaMemcpyAsync(h->O_keep, h->O, sizeof(float2) * h->HW, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(h->P_keep, h->P, sizeof(float2) * h->K, cudaMemcpyDeviceToDevice, h->st));
  }
  if (n == 0) {
    CK(cudaMemsetAsync(h->err_out + slot, 0, sizeof(double), h->st));
    return EPIE_OK;
  }
  std::vector<int32_t> order, gstart;
  make_order(h, h->sweep, n, order, gstart);
  if ((h->cfg.flags & EPIE_GRAPH) && h->cfg.path == EPIE_PATH_FUSED && !h->ktime)
    return run_sweep_graph(h, slot, order, gstart, kernels);
  CK(cudaMemcpyAsync(h->order_d, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, h->st));
  const int ng = static_cast<int>(gstart.size()) - 1;
  for (int g = 0; g < ng; ++g) {
    const int m = gstart[g + 1] - gstart[g];
    if (m == 0) continue;
    int rc = run_group(h, h->order_d + gstart[g], m, g > 0, kernels);
    if (rc) return rc;
  }
  CK(epie::launch_error_reduce(h->err_part, h->isum_part, n, h->err_stride, h->err_out + slot,
                               h->err_blocks, h->st));
  *kernels += 2;
  if (h->ktime && h->kev_used > 0) {
    CK(cudaEventSynchronize(h->kev[h->kev_used - 1]));
    for (int i = 0; i < h->kev_used; i += 2) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, h->kev[i], h->kev[i + 1]));
      h->kt_ms += ms;
      h->kt_launches += 1;
      h->kt_frames += h->kev_frames[i / 2];
    }
    h->kev_used = 0;
  }
  return EPIE_OK;
}

}  // namespace

// ------------------------------------------------------------------ ABI

extern "C" {

void epie_config_default(epie_config *c) {
  if (!c) return;
  std::memset(c, 0, sizeof *c);
  c->N = 256;
  c->obj_h = c->obj_w = 1024;
  c->capacity = 1024;
  c->intensity_dtype = EPIE_U16;
  c->mode = EPIE_COLOURED;
  c->batch = 64;
  c->omax_mode = EPIE_OMAX_PATCH;
  c->path = EPIE_PATH_FUSED;
  c->alpha = c->beta = 1.0f;
  c->seed = 0;
  c->device = 0;
  c->stream = nullptr;
  c->flags = 0;
  c->class_cap = 0;
  c->gemm_precision = EPIE_GEMM_BF16X3;
}

const char *epie_error(epie_t h) { return h ? h->err.c_str() : g_init_error.c_str(); }

int epie_destroy(epie_t h) {
  if (!h) return EPIE_OK;
  {
    CallLock lk(h);
    cudaSetDevice(h->cfg.device);
    if (h->st) cudaStreamSynchronize(h->st);
    if (h->up) cudaStreamSynchronize(h->up);
    for (auto &kv : h->plans) cufftDestroy(kv.second);
    epie::gemm_path_destroy(h->gemm);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    for (int b = 0; b < 2; ++b) {
      if (h->order_h[b]) cudaFreeHost(h->order_h[b]);
      if (h->gstart_h[b]) cudaFreeHost(h->gstart_h[b]);
      if (h->ev_order[b]) cudaEventDestroy(h->ev_order[b]);
    }
    void *dev[] = {h->gstart_d, h->err_sweep, h->O, h->P, h->twiddle, h->frames, h->pos_d, h->order_d, h->dark_d,
                   h->probe_part, h->err_part, h->err_blocks, h->isum_part, h->pmax2, h->omax_glob,
                   h->omax_tmp, h->err_out, h->flag_d, h->O_keep, h->P_keep, h->psi,
                   h->omax_m, h->accO, h->cnt, h->stage_d, h->amp, h->amp_isum};
    for (void *p : dev)
      if (p) cudaFree(p);
    for (void *p : h->stage_h)
      if (p) cudaFreeHost(p);
    if (h->err_h) cudaFreeHost(h->err_h);
    for (cudaEvent_t e : {h->ev_up, h->ev_st, h->ev_t0, h->ev_t1, h->ev_stage[0], h->ev_stage[1]})
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : h->kev) cudaEventDestroy(e);
    if (h->up) cudaStreamDestroy(h->up);
    if (h->own_stream && h->st) cudaStreamDestroy(h->st);
  }
  delete h;
  return EPIE_OK;
}

static int init_fail(epie_t h, int code) {
  g_init_error = h->err;
  epie_destroy(h);
  return code;
}

int epie_init(epie_t *out, const epie_config *cfg, const float *probe0, const float *object0) {
  if (!out) {
    g_init_error = "epie_init: out is NULL";
    return EPIE_EINVAL;
  }
  *out = nullptr;
  if (!cfg || !probe0) {
    g_init_error = "epie_init: cfg and probe0 are required";
    return EPIE_EINVAL;
  }
  const epie_config c = *cfg;
  std::string why;
  if (!(c.N == 64 || c.N == 128 || c.N == 256 || c.N == 512)) why = "N must be 64, 128, 256 or 512";
  else if (c.obj_h < c.N || c.obj_w < c.N) why = "object must be at least N x N";
  else if (static_cast<long long>(c.obj_h) * c.obj_w > (1LL << 31)) why = "object too large";
  else if (c.capacity < 0) why = "capacity must be >= 0";
  else if (c.intensity_dtype < EPIE_U16 || c.intensity_dtype > EPIE_F32) why = "bad intensity_dtype";
  else if (c.mode < EPIE_SEQUENTIAL || c.mode > EPIE_MINIBATCH) why = "bad mode";
  else if (c.mode == EPIE_MINIBATCH && c.batch < 1) why = "batch must be >= 1";
  else if (c.omax_mode != EPIE_OMAX_PATCH && c.omax_mode != EPIE_OMAX_GLOBAL) why = "bad omax_mode";
  else if (c.path < EPIE_PATH_FUSED || c.path > EPIE_PATH_GEMM) why = "bad path";
  else if (c.gemm_precision < EPIE_GEMM_BF16 || c.gemm_precision > EPIE_GEMM_TC_TF32X3)
    why = "bad gemm_precision";
  else if (!std::isfinite(c.alpha) || !std::isfinite(c.beta)) why = "alpha and beta must be finite";
  else if (c.flags & ~(EPIE_CHECKED | EPIE_PROBE_SUM | EPIE_GRAPH | EPIE_FRAMES_FFT_ORDER |
                       EPIE_RAW_INTENSITY))
    why = "unknown flags";
  else if (c.class_cap < 0) why = "class_cap must be >= 0";
  else if (c.path == EPIE_PATH_FUSED && epie::fused_ctas_per_frame(c.N, c.ctas_per_frame) == 0)
    why = "ctas_per_frame: tile shape not built for this N (0 = default; 1, 2, 4 at N = 128)";
  if (!why.empty()) {
    g_init_error = "epie_init: " + why;
    return EPIE_EINVAL;
  }
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev == 0) {
    g_init_error = std::string("epie_init: no CUDA device: ") + cudaGetErrorString(ce);
    return EPIE_ECUDA;
  }
  if (c.device < 0 || c.device >= ndev) {
    g_init_error = "epie_init: device ordinal out of range";
    return EPIE_EINVAL;
  }
  epie_t h = new epie_ctx;
  h->cfg = c;
  h->K = c.N * c.N;
  h->HW = static_cast<long long>(c.obj_h) * c.obj_w;
  // partial error slots per frame: one per CTA of the fused kernel, one per
  // block of the plain path's modulus kernel; every slot is written each sweep
  h->err_stride = c.path == EPIE_PATH_FUSED ? epie::fused_ctas_per_frame(c.N, c.ctas_per_frame)
                                            : epie::plain_err_stride(c.N);  // plain and GEMM
  h->cell_rows = (c.obj_h + c.N - 1) / c.N;
  h->cell_cols = (c.obj_w + c.N - 1) / c.N;
  h->cells.resize(static_cast<size_t>(h->cell_rows) * h->cell_cols);
  const int cap = std::max(c.capacity, 1);
  const size_t es = esize_of(c.intensity_dtype);
#define IK(expr)                                      \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) {                          \
      h->cuda_fail(e_, #expr);                        \
      return init_fail(h, EPIE_ECUDA);                \
    }                                                 \
  } while (0)
  IK(cudaSetDevice(c.device));
  if (c.stream) {
    h->st = static_cast<cudaStream_t>(c.stream);
  } else {
    IK(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  IK(cudaStreamCreateWithFlags(&h->up, cudaStreamNonBlocking));
  IK(cudaEventCreateWithFlags(&h->ev_up, cudaEventDisableTiming));
  IK(cudaEventCreateWithFlags(&h->ev_st, cudaEventDisableTiming));
  IK(cudaEventCreate(&h->ev_t0));
  IK(cudaEventCreate(&h->ev_t1));
  IK(cudaEventCreateWithFlags(&h->ev_stage[0], cudaEventDisableTiming));
  IK(cudaEventCreateWithFlags(&h->ev_stage[1], cudaEventDisableTiming));
  IK(cudaEventRecord(h->ev_up, h->up));
  IK(cudaMalloc(&h->O, sizeof(float2) * h->HW));
  IK(cudaMalloc(&h->P, sizeof(float2) * h->K));
  IK(cudaMalloc(&h->twiddle, sizeof(float2) * c.N));
  IK(cudaMalloc(&h->frames, es * h->K * static_cast<size_t>(cap)));
  IK(cudaMalloc(&h->pos_d, sizeof(int32_t) * 2 * static_cast<size_t>(cap)));
  IK(cudaMalloc(&h->order_d, sizeof(int32_t) * static_cast<size_t>(cap)));
  IK(cudaMalloc(&h->dark_d, sizeof(float) * h->K));
  if (c.path == EPIE_PATH_FUSED && !(c.flags & EPIE_RAW_INTENSITY)) {
    IK(cudaMalloc(&h->amp, sizeof(float) * h->K * static_cast<size_t>(cap)));
    IK(cudaMalloc(&h->amp_isum, sizeof(double) * static_cast<size_t>(cap)));
  }
  IK(cudaMalloc(&h->err_part, sizeof(double) * h->err_stride * static_cast<size_t>(cap)));
  IK(cudaMalloc(&h->err_blocks, sizeof(double) * 2 * epie::ERR_BLOCKS));
  IK(cudaMalloc(&h->isum_part, sizeof(double) * h->err_stride * static_cast<size_t>(cap)));
  IK(cudaMalloc(&h->pmax2, sizeof(unsigned long long) * 2));
  IK(cudaMalloc(&h->omax_glob, sizeof(double)));
  IK(cudaMalloc(&h->omax_tmp, sizeof(unsigned long long)));
  IK(cudaMalloc(&h->err_out, sizeof(double) * 1024));
  IK(cudaMallocHost(&h->err_h, sizeof(double) * 1024));
  IK(cudaMalloc(&h->flag_d, sizeof(int)));
  IK(cudaMalloc(&h->gstart_d, sizeof(int32_t) * (static_cast<size_t>(cap) + 1)));
  IK(cudaMalloc(&h->err_sweep, sizeof(double)));
  for (int b = 0; b < 2; ++b) {
    IK(cudaMallocHost(&h->order_h[b], sizeof(int32_t) * static_cast<size_t>(cap)));
    IK(cudaMallocHost(&h->gstart_h[b], sizeof(int32_t) * (static_cast<size_t>(cap) + 1)));
    IK(cudaEventCreateWithFlags(&h->ev_order[b], cudaEventDisableTiming));
    IK(cudaEventRecord(h->ev_order[b], h->st));
  }
  IK(cudaMemsetAsync(h->flag_d, 0, sizeof(int), h->st));
  IK(cudaMemsetAsync(h->pmax2, 0, sizeof(unsigned long long) * 2, h->st));
  if (c.flags & EPIE_CHECKED) {
    IK(cudaMalloc(&h->O_keep, sizeof(float2) * h->HW));
    IK(cudaMalloc(&h->P_keep, sizeof(float2) * h->K));
  }
  if (c.mode == EPIE_MINIBATCH) {
    IK(cudaMalloc(&h->accO, sizeof(float2) * h->HW));
    IK(cudaMalloc(&h->cnt, sizeof(int) * h->HW));
    IK(cudaMemsetAsync(h->accO, 0, sizeof(float2) * h->HW, h->st));
    IK(cudaMemsetAsync(h->cnt, 0, sizeof(int) * h->HW, h->st));
  }
  {
    const int pre = c.mode == EPIE_MINIBATCH ? c.batch : (c.mode == EPIE_SEQUENTIAL ? 1 : 64);
    if (ensure_part(h, pre) != EPIE_OK) return init_fail(h, EPIE_ECUDA);
  }
  // staging: two pinned host buffers and one device buffer of whole frames
  {
    const size_t frame_bytes = es * h->K;
    const size_t want = std::max<size_t>(frame_bytes, (size_t)64 << 20);
    h->stage_bytes = want / frame_bytes * frame_bytes;
    IK(cudaMallocHost(&h->stage_h[0], h->stage_bytes));
    IK(cudaMallocHost(&h->stage_h[1], h->stage_bytes));
    IK(cudaMalloc(&h->stage_d, h->stage_bytes));
    IK(cudaEventRecord(h->ev_stage[0], h->up));
    IK(cudaEventRecord(h->ev_stage[1], h->up));
  }
  // twiddles exp(-2 pi i m / N), evaluated in double precision on the host
  {
    std::vector<float2> tw(c.N);
    for (int m = 0; m < c.N; ++m) {
      const double ang = -2.0 * 3.14159265358979323846 * m / c.N;
      tw[m] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
    }
    IK(cudaMemcpy(h->twiddle, tw.data(), sizeof(float2) * c.N, cudaMemcpyHostToDevice));
  }
  IK(cudaMemcpy(h->P, probe0, sizeof(float2) * h->K, cudaMemcpyHostToDevice));
  if (object0) {
    IK(cudaMemcpy(h->O, object0, sizeof(float2) * h->HW, cudaMemcpyHostToDevice));
  } else {
    IK(epie::launch_fill(h->O, h->HW, make_float2(1.f, 0.f), h->st));
  }
  if (c.path == EPIE_PATH_GEMM) {
    std::string why;
    h->gemm = epie::gemm_path_create(c.N, c.gemm_precision, h->st, &why);
    if (!h->gemm) {
      h->err = "epie_init: " + why;
      return init_fail(h, EPIE_ECUDA);
    }
  }
  if (recompute_pmax(h) != EPIE_OK) return init_fail(h, EPIE_ECUDA);
  IK(cudaStreamSynchronize(h->st));
#undef IK
  *out = h;
  return EPIE_OK;
}

int epie_set_dark(epie_t h, const float *dark) {
  int rc = check_handle(h);
  if (rc) return rc;
  CallLock lk(h);
  CK(cudaSetDevice(h->cfg.device));
  CK(cudaStreamWaitEvent(h->st, h->ev_up, 0));
  if (dark) {
    float *tmp = reinterpret_cast<float *>(h->stage_d);
    if (h->cfg.flags & EPIE_FRAMES_FFT_ORDER) {
      CK(cudaMemcpyAsync(h->dark_d, dark, sizeof(float) * h->K, cudaMemcpyHostToDevice, h->st));
    } else {
      CK(cudaMemcpyAsync(tmp, dark, sizeof(float) * h->K, cudaMemcpyHostToDevice, h->st));
      CK(epie::launch_dark_ingest(tmp, h->dark_d, h->cfg.N, h->st));
      h->launches_total += 1;
    }
  }
  h->has_dark = dark != nullptr;
  if (h->amp && h->n_frames > 0) {  // the frames' amplitudes follow the dark field
    CK(epie::launch_amp_ingest(h->frames, h->cfg.intensity_dtype, h->has_dark ? h->dark_d : nullptr,
                               h->amp, h->amp_isum, 0, h->n_frames, h->cfg.N, h->cfg.ctas_per_frame, h->st));
    h->launches_total += 1;
  }
  CK(cudaStreamSynchronize(h->st));
  return EPIE_OK;
}

static int append_impl(epie_t h, const void *frames, const int32_t *pos, int32_t n, bool device) {
  int rc = check_handle(h);
  if (rc) return rc;
  CallLock lk(h);
  if (n < 0 || (n > 0 && (!frames || !pos))) return h->fail(EPIE_EINVAL, "append: bad arguments");
  if (n == 0) return EPIE_OK;
  const int N = h->cfg.N;
  if (static_cast<long long>(h->n_frames) + n > h->cfg.capacity)
    return h->fail(EPIE_ECAPACITY, "append: %d + %d frames exceed capacity %d", h->n_frames, n,
                   h->cfg.capacity);
  for (int32_t i = 0; i < n; ++i) {
    const int y = pos[2 * i], x = pos[2 * i + 1];
    if (y < 0 || x < 0 || y > h->cfg.obj_h - N || x > h->cfg.obj_w - N)
      return h->fail(EPIE_ERANGE, "append: frame %d at (%d, %d) leaves the %d x %d object", i, y,
                     x, h->cfg.obj_h, h->cfg.obj_w);
  }
  CK(cudaSetDevice(h->cfg.device));
  // Sweeps queued on st may still read the slots this append writes (after
  // a truncation, the frames and positions past n_keep): the upload stream
  // waits for everything queued on st so far.
  CK(cudaEventRecord(h->ev_st, h->st));
  CK(cudaStreamWaitEvent(h->up, h->ev_st, 0));
  const size_t es = esize_of(h->cfg.intensity_dtype);
  const size_t fb = es * h->K;
  const int per = static_cast<int>(h->stage_bytes / fb);
  char *dst0 = static_cast<char *>(h->frames) + fb * static_cast<size_t>(h->n_frames);
  bool pinned = false;
  if (!device) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, frames) == cudaSuccess && at.type == cudaMemoryTypeHost)
      pinned = true;
    else
      cudaGetLastError();
  }
  // frames already in FFT order go straight to the frame set; DC-centred
  // frames pass through the staging buffer and the re-layout kernel
  const bool fft_order = (h->cfg.flags & EPIE_FRAMES_FFT_ORDER) != 0;
  for (int32_t a = 0; a < n; a += per) {
    const int m = std::min(per, n - a);
    const char *src = static_cast<const char *>(frames) + fb * static_cast<size_t>(a);
    char *dst = dst0 + fb * static_cast<size_t>(a);
    char *to = fft_order ? dst : static_cast<char *>(h->stage_d);
    if (device || pinned) {
      // device or page-locked source: one copy
      CK(cudaMemcpyAsync(to, src, fb * m,
                         device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->up));
    } else {
      const int b = h->stage_next;
      h->stage_next ^= 1;
      CK(cudaEventSynchronize(h->ev_stage[b]));  // buffer b free again
      std::memcpy(h->stage_h[b], src, fb * m);
      CK(cudaMemcpyAsync(to, h->stage_h[b], fb * m, cudaMemcpyHostToDevice, h->up));
      CK(cudaEventRecord(h->ev_stage[b], h->up));
    }
    if (!fft_order) {
      CK(epie::launch_ingest(h->stage_d, dst, m, N, static_cast<int>(es), h->up));
      h->launches_total += 1;
    }
  }
  if (h->amp) {
    CK(epie::launch_amp_ingest(h->frames, h->cfg.intensity_dtype,
                               h->has_dark ? h->dark_d : nullptr, h->amp, h->amp_isum,
                               h->n_frames, n, N, h->cfg.ctas_per_frame, h->up));
    h->launches_total += 1;
  }
  CK(cudaMemcpyAsync(h->pos_d + 2 * static_cast<size_t>(h->n_frames), pos,
                     sizeof(int32_t) * 2 * n, cudaMemcpyHostToDevice, h->up));
  CK(cudaEventRecord(h->ev_up, h->up));
  // the caller's buffer must be free when we return
  CK(cudaStreamSynchronize(h->up));
  const int32_t f0 = h->n_frames;
  h->pos_h.insert(h->pos_h.end(), pos, pos + 2 * static_cast<size_t>(n));
  h->colour.resize(static_cast<size_t>(f0) + n);
  for (int32_t i = 0; i < n; ++i) colour_append(h, f0 + i);
  h->n_frames = f0 + n;
  return EPIE_OK;
}

int epie_append_frames(epie_t h, const void *frames, const int32_t *pos_yx, int32_t n) {
  return append_impl(h, frames, pos_yx, n, false);
}

int epie_append_frames_device(epie_t h, const void *frames_dev, const int32_t *pos_yx, int32_t n) {
  return append_impl(h, frames_dev, pos_yx, n, true);
}

int epie_truncate_frames(epie_t h, int32_t n_keep) {
  int rc = check_handle(h);
  if (rc) return rc;
  CallLock lk(h);
  if (n_keep < 0 || n_keep > h->n_frames)
    return h->fail(EPIE_EINVAL, "truncate: n_keep %d outside [0, %d]", n_keep, h->n_frames);
  const int N = h->cfg.N;
  for (int32_t f = h->n_frames - 1; f >= n_keep; --f) {
    // the newest frame is last in its class and in its grid cell
    h->classes[h->colour[f]].pop_back();
    const int cy = h->pos_h[2 * f] / N, cx = h->pos_h[2 * f + 1] / N;
    h->cells[static_cast<size_t>(cy) * h->cell_cols + cx].pop_back();
  }
  while (!h->classes.empty() && h->classes.back().empty()) {
    h->classes.pop_back();
    h->stamp.pop_back();
  }
  h->pos_h.resize(2 * static_cast<size_t>(n_keep));
  h->colour.resize(n_keep);
  h->n_frames = n_keep;
  return EPIE_OK;
}

// Reads the errors of sweeps [s0, s0 + cnt) of this call from slots [first,
// first + cnt), checks the device status word and non-finite errors (with
// EPIE_CHECKED restoring the sweep start).  Call with h->mu held.
static int fetch_errors(epie_t h, int first, int cnt, int32_t s0, double *err_per_sweep) {
  CK(cudaMemcpyAsync(h->err_h + first, h->err_out + first, sizeof(double) * cnt,
                     cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  int flag = 0;
  CK(cudaMemcpy(&flag, h->flag_d, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) return h->fail(EPIE_ETIMEOUT, "a bounded device wait expired (flag %d)", flag);
  for (int i = 0; i < cnt; ++i) {
    const double e = h->err_h[first + i];
    if (err_per_sweep) err_per_sweep[s0 + i] = e;
    if (!std::isfinite(e))
      return h->fail(EPIE_ENUMERIC, "sweep %lld: error metric is not finite",
                     static_cast<long long>(h->sweep - cnt + i + 1));
  }
  return EPIE_OK;
}

int epie_iterate_many(epie_t *hs, int32_t k, int32_t n_sweeps, double *err) {
  if (!hs || k < 0 || n_sweeps < 0) {
    g_init_error = "epie_iterate_many: bad arguments";
    return EPIE_EINVAL;
  }
  for (int32_t i = 0; i < k; ++i) {
    int rc = check_handle(hs[i]);
    if (rc) return rc;
    if (hs[i]->cfg.flags & EPIE_CHECKED)
      return hs[i]->fail(EPIE_EINVAL, "epie_iterate_many: EPIE_CHECKED handles need epie_iterate");
    for (int32_t j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return hs[i]->fail(EPIE_EINVAL, "epie_iterate_many: handle repeated");
  }
  int first_rc = EPIE_OK;
  std::vector<int> failed(k, 0);
  for (int32_t c0 = 0; c0 < n_sweeps; c0 += 1024) {
    const int32_t cn = std::min<int32_t>(1024, n_sweeps - c0);
    for (int32_t s = 0; s < cn; ++s)
      for (int32_t i = 0; i < k; ++i) {
        if (failed[i]) continue;
        epie_t h = hs[i];
        CallLock lk(h);
        int64_t kern = 0;
        int rc = cudaSetDevice(h->cfg.device) == cudaSuccess ? EPIE_OK
                                                             : h->fail(EPIE_ECUDA, "cudaSetDevice");
        if (!rc) rc = run_sweep(h, s, &kern);
        if (!rc) {
          h->sweep += 1;
          h->launches_total += kern;
        }
        if (rc) {
          failed[i] = 1;
          if (!first_rc) first_rc = rc;
        }
      }
    for (int32_t i = 0; i < k; ++i) {
      if (failed[i]) continue;
      epie_t h = hs[i];
      CallLock lk(h);
      int rc = fetch_errors(h, 0, cn, c0, err ? err + static_cast<size_t>(i) * n_sweeps : nullptr);
      if (rc) {
        failed[i] = 1;
        if (!first_rc) first_rc = rc;
      }
    }
  }
  return first_rc;
}

int epie_average_state(epie_t *hs, int32_t k) {
  if (!hs || k < 1) {
    g_init_error = "epie_average_state: bad arguments";
    return EPIE_EINVAL;
  }
  for (int32_t i = 0; i < k; ++i) {
    int rc = check_handle(hs[i]);
    if (rc) return rc;
    const epie_config &a = hs[0]->cfg, &b = hs[i]->cfg;
    if (a.N != b.N || a.obj_h != b.obj_h || a.obj_w != b.obj_w || a.device != b.device)
      return hs[i]->fail(EPIE_EINVAL, "epie_average_state: handles differ in N, object or device");
    for (int32_t j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return hs[i]->fail(EPIE_EINVAL, "epie_average_state: handle repeated");
  }
  if (k == 1) return EPIE_OK;
  std::vector<std::unique_lock<std::mutex>> locks;
  for (int32_t i = 0; i < k; ++i) locks.emplace_back(hs[i]->mu);
  epie_t h = hs[0];
  CK(cudaSetDevice(h->cfg.device));
  for (int32_t i = 0; i < k; ++i) CK(cudaStreamSynchronize(hs[i]->st));
  // source pointer tables: objects, then probes
  std::vector<const float2 *> tab(2 * static_cast<size_t>(k));
  for (int32_t i = 0; i < k; ++i) {
    tab[i] = hs[i]->O;
    tab[k + i] = hs[i]->P;
  }
  const float2 **tab_d = nullptr;
  CK(cudaMalloc(&tab_d, sizeof(float2 *) * tab.size()));
  cudaError_t e = cudaMemcpy(tab_d, tab.data(), sizeof(float2 *) * tab.size(),
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = epie::launch_average(tab_d, k, h->O, h->HW, h->st);
  if (e == cudaSuccess) e = epie::launch_average(tab_d + k, k, h->P, h->K, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  cudaFree(tab_d);
  if (e != cudaSuccess) return h->cuda_fail(e, "epie_average_state");
  for (int32_t i = 1; i < k; ++i) {
    CK(cudaMemcpyAsync(hs[i]->O, h->O, sizeof(float2) * h->HW, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(hs[i]->P, h->P, sizeof(float2) * h->K, cudaMemcpyDeviceToDevice, h->st));
  }
  CK(cudaStreamSynchronize(h->st));
  for (int32_t i = 0; i < k; ++i) {
    int rc = recompute_pmax(hs[i]);
    if (rc) return rc;
    CK(cudaStreamSynchronize(hs[i]->st));
  }
  h->launches_total += 2;
  return EPIE_OK;
}

int epie_iterate(epie_t h, int32_t n_sweeps, double *err_per_sweep) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (n_sweeps < 0) return h->fail(EPIE_EINVAL, "iterate: n_sweeps < 0");
  int64_t kernels = 0;
  {
    std::lock_guard<std::mutex> lk(h->mu);
    CK(cudaSetDevice(h->cfg.device));
    CK(cudaEventRecord(h->ev_t0, h->st));
    h->iter_frames.clear();
  }
  for (int32_t s = 0; s < n_sweeps; ++s) {
    // Calls from other threads (a feeder's append) slip in between sweeps:
    // while one is waiting for the mutex, hand it over instead of re-taking
    // it at once (bounded, so a stream of calls cannot stall the sweeps).
    for (int spin = 0; h->waiting.load() > 0 && spin < 100000; ++spin) std::this_thread::yield();
    std::lock_guard<std::mutex> lk(h->mu);
    if (h->dead) return h->fail(EPIE_ESTATE, "handle unusable: %s", h->err.c_str());
    const int slot = s % 1024;
    h->iter_frames.push_back(h->n_frames);
    rc = run_sweep(h, slot, &kernels);
    if (rc) return rc;
    h->sweep += 1;
    const bool last = s + 1 == n_sweeps;
    if (last || slot == 1023 || (h->cfg.flags & EPIE_CHECKED)) {
      // fetch the errors of this chunk of sweeps and the device status word
      // slots [first, slot] hold sweeps s - (slot - first) .. s of this call
      const int first = (h->cfg.flags & EPIE_CHECKED) ? slot : 0;
      const int cnt = slot - first + 1;
      CK(cudaMemcpyAsync(h->err_h + first, h->err_out + first, sizeof(double) * cnt,
                         cudaMemcpyDeviceToHost, h->st));
      int flag = 0;
      CK(cudaStreamSynchronize(h->st));
      CK(cudaMemcpy(&flag, h->flag_d, sizeof(int), cudaMemcpyDeviceToHost));
      if (flag) return h->fail(EPIE_ETIMEOUT, "a bounded device wait expired (flag %d)", flag);
      for (int i = first; i <= slot; ++i) {
        const int32_t sw = s - (slot - i);
        const double e = h->err_h[i];
        if (err_per_sweep) err_per_sweep[sw] = e;
        if (!std::isfinite(e)) {
          if (h->cfg.flags & EPIE_CHECKED) {
            CK(cudaMemcpyAsync(h->O, h->O_keep, sizeof(float2) * h->HW, cudaMemcpyDeviceToDevice,
                               h->st));
            CK(cudaMemcpyAsync(h->P, h->P_keep, sizeof(float2) * h->K, cudaMemcpyDeviceToDevice,
                               h->st));
            if ((rc = recompute_pmax(h))) return rc;
            CK(cudaStreamSynchronize(h->st));
            h->sweep -= 1;
          }
          return h->fail(EPIE_ENUMERIC, "sweep %lld: error metric is not finite",
                         static_cast<long long>(h->sweep));
        }
      }
    }
  }
  std::lock_guard<std::mutex> lk(h->mu);
  CK(cudaEventRecord(h->ev_t1, h->st));
  CK(cudaEventSynchronize(h->ev_t1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1));
  h->last_ms = ms;
  h->last_kernels = kernels;
  h->launches_total += kernels;
  return EPIE_OK;
}

static int copy_state(epie_t h, void *host, const void *dev, size_t bytes, size_t want_floats,
                      size_t n_floats, bool to_dev, const char *what) {
  int rc = check_handle(h);
  if (rc) return rc;
  CallLock lk(h);
  if (!host || n_floats != want_floats)
    return h->fail(EPIE_EINVAL, "%s: need %zu floats, got %zu", what, want_floats, n_floats);
  CK(cudaSetDevice(h->cfg.device));
  CK(cudaStreamSynchronize(h->st));
  if (to_dev) {
    CK(cudaMemcpy(const_cast<void *>(dev), host, bytes, cudaMemcpyHostToDevice));
  } else {
    CK(cudaMemcpy(host, dev, bytes, cudaMemcpyDeviceToHost));
  }
  return EPIE_OK;
}

int epie_get_object(epie_t h, float *dst, size_t n_floats) {
  if (!h) return EPIE_EINVAL;
  return copy_state(h, dst, h->O, sizeof(float2) * h->HW, 2 * static_cast<size_t>(h->HW), n_floats,
                    false, "get_object");
}

int epie_get_probe(epie_t h, float *dst, size_t n_floats) {
  if (!h) return EPIE_EINVAL;
  return copy_state(h, dst, h->P, sizeof(float2) * h->K, 2 * static_cast<size_t>(h->K), n_floats,
                    false, "get_probe");
}

int epie_set_object(epie_t h, const float *src, size_t n_floats) {
  if (!h) return EPIE_EINVAL;
  return copy_state(h, const_cast<float *>(src), h->O, sizeof(float2) * h->HW,
                    2 * static_cast<size_t>(h->HW), n_floats, true, "set_object");
}

int epie_set_probe(epie_t h, const float *src, size_t n_floats) {
  if (!h) return EPIE_EINVAL;
  int rc = copy_state(h, const_cast<float *>(src), h->P, sizeof(float2) * h->K,
                      2 * static_cast<size_t>(h->K), n_floats, true, "set_probe");
  if (rc) return rc;
  CallLock lk(h);
  if ((rc = recompute_pmax(h))) return rc;
  CK(cudaStreamSynchronize(h->st));
  return EPIE_OK;
}

int epie_num_frames(epie_t h, int32_t *n) {
  if (!h || !n) return EPIE_EINVAL;
  CallLock lk(h);
  *n = h->n_frames;
  return EPIE_OK;
}

int epie_num_classes(epie_t h, int32_t *n) {
  if (!h || !n) return EPIE_EINVAL;
  CallLock lk(h);
  *n = static_cast<int32_t>(h->classes.size());
  return EPIE_OK;
}

int epie_get_colours(epie_t h, int32_t *colour, int32_t n) {
  if (!h || (!colour && n > 0)) return EPIE_EINVAL;
  CallLock lk(h);
  if (n < 0 || n > h->n_frames) return h->fail(EPIE_EINVAL, "get_colours: bad count %d", n);
  std::copy(h->colour.begin(), h->colour.begin() + n, colour);
  return EPIE_OK;
}

int epie_get_order(epie_t h, int64_t sweep, int32_t *order, int32_t *group_start,
                   int32_t *n_groups) {
  if (!h || !n_groups) return EPIE_EINVAL;
  CallLock lk(h);
  if (h->n_frames > 0 && (!order || !group_start))
    return h->fail(EPIE_EINVAL, "get_order: NULL output");
  std::vector<int32_t> o, g;
  make_order(h, sweep, h->n_frames, o, g);
  std::copy(o.begin(), o.end(), order);
  std::copy(g.begin(), g.end(), group_start);
  *n_groups = static_cast<int32_t>(g.size()) - 1;
  return EPIE_OK;
}

int epie_get_sweep_index(epie_t h, int64_t *sweep) {
  if (!h || !sweep) return EPIE_EINVAL;
  CallLock lk(h);
  *sweep = h->sweep;
  return EPIE_OK;
}

int epie_set_sweep_index(epie_t h, int64_t sweep) {
  if (!h || sweep < 0) return EPIE_EINVAL;
  CallLock lk(h);
  h->sweep = sweep;
  return EPIE_OK;
}

int epie_last_timing(epie_t h, double *ms, int64_t *kernels) {
  if (!h) return EPIE_EINVAL;
  CallLock lk(h);
  if (ms) *ms = h->last_ms;
  if (kernels) *kernels = h->last_kernels;
  return EPIE_OK;
}

int epie_frames_to_fft_order(const void *src, void *dst, int32_t n, int32_t N,
                             int32_t intensity_dtype, void *stream) {
  if (!(N == 64 || N == 128 || N == 256 || N == 512) || n < 0 || (n > 0 && (!src || !dst)) ||
      intensity_dtype < EPIE_U16 || intensity_dtype > EPIE_F32) {
    g_init_error = "epie_frames_to_fft_order: bad arguments";
    return EPIE_EINVAL;
  }
  cudaError_t e = epie::launch_ingest(src, dst, n, N, static_cast<int>(esize_of(intensity_dtype)),
                                      static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    g_init_error = std::string("epie_frames_to_fft_order: ") + cudaGetErrorString(e);
    return EPIE_ECUDA;
  }
  return EPIE_OK;
}

int epie_tc_gemm_bf16(const void *A0, const void *A1, const void *B0, const void *B1, float *D,
                      int64_t M, int32_t Nn, int32_t K, int32_t ldd, int32_t terms,
                      int32_t *status, void *stream) {
  std::string why;
  const int rc = epie::tc_gemm_bf16(A0, A1, B0, B1, D, M, Nn, K, ldd, terms, status,
                                    static_cast<cudaStream_t>(stream), &why);
  if (rc) g_init_error = "epie_tc_gemm_bf16: " + why;
  return rc;
}

int epie_tc_gemm_tf32(const float *A0, const float *A1, const float *B0, const float *B1,
                      float *D, int64_t M, int32_t Nn, int32_t K, int32_t ldd, int32_t terms,
                      int32_t *status, void *stream) {
  std::string why;
  const int rc = epie::tc_gemm_tf32(A0, A1, B0, B1, D, M, Nn, K, ldd, terms, status,
                                    static_cast<cudaStream_t>(stream), &why);
  if (rc) g_init_error = "epie_tc_gemm_tf32: " + why;
  return rc;
}

int epie_fp32_fma_peak(int32_t device, int32_t iters, double *tflops, double *sm_mhz) {
  if (iters < 1 || !tflops || !sm_mhz) {
    g_init_error = "epie_fp32_fma_peak: iters must be >= 1 and the outputs non-NULL";
    return EPIE_EINVAL;
  }
  std::string why;
  const int rc = epie::fma_peak(device, iters, tflops, sm_mhz, &why);
  if (rc) g_init_error = "epie_fp32_fma_peak: " + why;
  return rc;
}

int epie_last_sweep_frames(epie_t h, int32_t *counts, int32_t cap, int32_t *n_out) {
  if (!h || !n_out || cap < 0 || (cap > 0 && !counts)) return EPIE_EINVAL;
  CallLock lk(h);
  const int32_t n = static_cast<int32_t>(h->iter_frames.size());
  *n_out = n;
  for (int32_t i = 0; i < std::min(n, cap); ++i) counts[i] = h->iter_frames[i];
  return EPIE_OK;
}

int epie_inject_fault(epie_t h, int32_t what, int32_t count, int64_t wait_ns) {
  if (count < 0 || wait_ns < 1000 || wait_ns > 2000000000LL) {
    g_init_error = "epie_inject_fault: count >= 0 and wait_ns in [1e3, 2e9] required";
    return EPIE_EINVAL;
  }
  if (what == EPIE_INJECT_TC_COPY) {
    epie::tc_gemm_inject(count, wait_ns);
    return EPIE_OK;
  }
  if (what != EPIE_INJECT_STEP_COPY || !h) {
    g_init_error = "epie_inject_fault: unknown kind, or no handle for EPIE_INJECT_STEP_COPY";
    return EPIE_EINVAL;
  }
  CallLock lk(h);
  if (h->cfg.path != EPIE_PATH_FUSED || (h->cfg.flags & EPIE_GRAPH))
    return h->fail(EPIE_EINVAL, "epie_inject_fault: step injection needs the fused path without "
                                "EPIE_GRAPH");
  h->inject_steps = count;
  h->inject_wait_ns = static_cast<unsigned long long>(wait_ns);
  return EPIE_OK;
}

int epie_launch_count(epie_t h, int64_t *total) {
  if (!h || !total) return EPIE_EINVAL;
  CallLock lk(h);
  *total = h->launches_total;
  return EPIE_OK;
}

int epie_set_kernel_timing(epie_t h, int32_t on) {
  if (!h) return EPIE_EINVAL;
  CallLock lk(h);
  h->ktime = on != 0;
  h->kev_used = 0;
  return EPIE_OK;
}

int epie_kernel_timing(epie_t h, int64_t *launches, double *ms, int64_t *frames) {
  if (!h) return EPIE_EINVAL;
  CallLock lk(h);
  if (launches) *launches = h->kt_launches;
  if (ms) *ms = h->kt_ms;
  if (frames) *frames = h->kt_frames;
  h->kt_launches = h->kt_frames = 0;
  h->kt_ms = 0.0;
  return EPIE_OK;
}

}  // extern "C"
