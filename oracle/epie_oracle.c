/*
 * epie_oracle.c -- plain, slow, FP64 CPU oracle for the ePIE hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the package's smoke check and
 * the timed CPU-baseline leg of the benchmark are the only code allowed to
 * load this library.  The product path (the CUDA library behind
 * include/epie.h and its Python binding) never calls, links or imports it,
 * and this file shares no code, header, table or constant generator with it.
 *
 * What is computed, and where it comes from:
 *   - ePIE (Maiden & Rodenburg 2009), the algorithm the paper's engine runs
 *     (Sec. "ePIE Implementation"): exit wave psi = P * O_j, far field
 *     Psi = F psi, modulus replacement Psi' = sqrt(I) Psi/|Psi|,
 *     psi' = F^-1 Psi', and simultaneous object / illumination updates with
 *     strengths alpha and beta (the paper uses alpha = beta = 1).
 *   - DFT forward / back projection on 2^n frames (same section): an own
 *     iterative radix-2 FFT with every twiddle evaluated directly as
 *     cos/sin(2 pi k / len) in double precision, plus an O(N^4) brute DFT.
 *   - Random shuffled visiting order per iteration (same section), drawn
 *     with SplitMix64 (Steele, Lea & Flood 2014) and Fisher-Yates.
 *   - Live extension of the frame set between sweeps (Sec. "Extensions of
 *     the ePIE implementation", "Simulating live and parallel processing"):
 *     every sweep covers the frames present when it starts.
 *   - Parallel averaging over disjoint subsets (Sec. "Simulating live and
 *     parallel processing") is composed from these sweeps in oracle.py.
 * Readings where the paper is silent (the engine takes the same ones):
 *   R1 F is the unnormalised DFT with exp(-2 pi i k.r/N); F^-1 carries 1/N^2.
 *      Frames arrive DC-centred; the DC moves to index 0 by ifftshift.
 *   R2 u(0) = 1: at |Psi| = 0 the replaced value is sqrt(I).
 *   R3 Object and probe updates of one step both use the pre-step P and O_j.
 *   R4 max|O|^2 is taken over the patch O_j by default, or over the whole
 *      object at group start (omax_global).  A zero maximum turns the
 *      corresponding update off (0/0 := 0).
 *   R5 Intensities below 0 after dark subtraction, and NaN, are clamped to 0.
 *   R6 Coloured sweep: greedy first-fit colour classes in append order
 *      (optionally capped in size: a full class is skipped);
 *      members of a class share the probe at class start; the probe moves
 *      by the mean (or sum) of the members' probe updates.
 *   R7 Mini-batch sweep: a batch of consecutive positions of the shuffled
 *      order shares the batch-start O and P; object updates are divided by
 *      the per-pixel count of covering patches, probe updates averaged.
 *   R8 Error metric E = sum_j sum_k (|Psi_j| - sqrt(I_j))^2 / sum_j sum_k I_j.
 *   R9 Order stream of sweep s: SplitMix64 state seed ^ (s * 0xD1B54A32D192ED03),
 *      Fisher-Yates with j = next() mod (i+1) for i = n-1 .. 1.
 *
 * Parity pins: see tests/test_oracle_pins.py.  The amplitude-loss gradient
 * (orc_amp_loss_grad) is pinned by central finite differences.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* complex.h defines I as the imaginary unit; the intensity is called I here */
#undef I

typedef double complex cplx;

#define ORC_PI 3.14159265358979323846264338327950288

static cplx mkc(double re, double im) { return CMPLX(re, im); }

/* ------------------------------------------------------------------------ */
/* DFT / FFT                                                                 */
/* ------------------------------------------------------------------------ */

/* In-place radix-2 FFT of n points at x[0], x[stride], ... ;
 * sign = -1 forward (exp(-2 pi i ...)), +1 backward (no scaling here). */
static void fft1(cplx *x, int n, long stride, int sign) {
  /* bit-reversal permutation */
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      cplx t = x[(long)i * stride];
      x[(long)i * stride] = x[(long)j * stride];
      x[(long)j * stride] = t;
    }
  }
  for (int len = 2; len <= n; len <<= 1) {
    int half = len / 2;
    for (int k = 0; k < half; ++k) {
      double ang = (double)sign * 2.0 * ORC_PI * (double)k / (double)len;
      cplx w = mkc(cos(ang), sin(ang));
      for (int i = 0; i < n; i += len) {
        cplx u = x[(long)(i + k) * stride];
        cplx v = x[(long)(i + k + half) * stride] * w;
        x[(long)(i + k) * stride] = u + v;
        x[(long)(i + k + half) * stride] = u - v;
      }
    }
  }
}

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* 2-D FFT of an n x n row-major array (R1).  sign -1: forward, unnormalised.
 * sign +1: inverse including the 1/n^2 factor. */
int orc_fft2(cplx *a, int n, int sign) {
  if (!is_pow2(n) || (sign != -1 && sign != 1)) return -1;
  for (int r = 0; r < n; ++r) fft1(a + (long)r * n, n, 1, sign);
  for (int c = 0; c < n; ++c) fft1(a + c, n, n, sign);
  if (sign == 1) {
    double s = 1.0 / ((double)n * (double)n);
    for (long i = 0; i < (long)n * n; ++i) a[i] *= s;
  }
  return 0;
}

/* Brute-force 2-D DFT from its definition, O(n^4), any n >= 1 (pins only). */
int orc_dft2_brute(const cplx *in, cplx *out, int n, int sign) {
  if (n < 1 || (sign != -1 && sign != 1)) return -1;
  for (int ky = 0; ky < n; ++ky)
    for (int kx = 0; kx < n; ++kx) {
      cplx acc = 0;
      for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
          /* reduce the phase index exactly in integers before the trig call */
          long m = ((long)ky * y + (long)kx * x) % n;
          double ang = (double)sign * 2.0 * ORC_PI * (double)m / (double)n;
          acc += in[(long)y * n + x] * mkc(cos(ang), sin(ang));
        }
      if (sign == 1) acc /= (double)n * (double)n;
      out[(long)ky * n + kx] = acc;
    }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Intensities: dequantisation, DC shift, dark subtraction (R1, R5)          */
/* ------------------------------------------------------------------------ */

/* IEEE binary16 bits -> double, from the format's definition. */
static double half_to_double(uint16_t h) {
  int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
  double v;
  if (e == 0) v = ldexp((double)m, -24);
  else if (e == 31) v = m ? NAN : INFINITY;
  else v = ldexp((double)(m | 1024), e - 25);
  return s ? -v : v;
}

/* frames: n frames of N*N values, DC-centred detector layout, dtype
 * 0 = uint16, 1 = binary16, 2 = float32.  dark: N*N float32 in the same
 * layout, or NULL.  out: n*N*N doubles in FFT order (DC at [0,0]):
 * out[ky,kx] = max(raw[(ky+N/2)%N, (kx+N/2)%N] - dark[...], 0). */
int orc_prepare_intensity(const void *frames, int dtype, long n, int N,
                          const float *dark, double *out) {
  if (!is_pow2(N) || n < 0) return -1;
  const long K = (long)N * N;
  for (long f = 0; f < n; ++f)
    for (int ky = 0; ky < N; ++ky)
      for (int kx = 0; kx < N; ++kx) {
        long src = (long)((ky + N / 2) % N) * N + (kx + N / 2) % N;
        double v;
        if (dtype == 0) v = ((const uint16_t *)frames)[f * K + src];
        else if (dtype == 1) v = half_to_double(((const uint16_t *)frames)[f * K + src]);
        else if (dtype == 2) v = ((const float *)frames)[f * K + src];
        else return -1;
        if (dark) v -= (double)dark[src];
        out[f * K + (long)ky * N + kx] = v > 0.0 ? v : 0.0;
      }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Modulus projection (ePIE, R2)                                             */
/* ------------------------------------------------------------------------ */

/* Psi <- sqrt(I) * Psi/|Psi| (sqrt(I) where |Psi| = 0).  Adds
 * sum (|Psi| - sqrt(I))^2 to *err and sum I to *isum when they are non-NULL. */
void orc_modulus_project(cplx *Psi, const double *I, long K, double *err, double *isum) {
  double e = 0.0, s = 0.0;
  for (long k = 0; k < K; ++k) {
    double a = cabs(Psi[k]);
    double r = sqrt(I[k] > 0.0 ? I[k] : 0.0);
    e += (a - r) * (a - r);
    s += I[k];
    Psi[k] = (a > 0.0) ? Psi[k] * (r / a) : mkc(r, 0.0);
  }
  if (err) *err += e;
  if (isum) *isum += s;
}

/* ------------------------------------------------------------------------ */
/* One ePIE position update (R3, R4)                                         */
/* ------------------------------------------------------------------------ */

static double max_abs2(const cplx *a, long n) {
  double m = 0.0;
  for (long i = 0; i < n; ++i) {
    double v = creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    if (v > m) m = v;
  }
  return m;
}

static double max_abs2_patch(const cplx *O, int W, int y0, int x0, int N) {
  double m = 0.0;
  for (int y = 0; y < N; ++y)
    for (int x = 0; x < N; ++x) {
      cplx o = O[(long)(y0 + y) * W + x0 + x];
      double v = creal(o) * creal(o) + cimag(o) * cimag(o);
      if (v > m) m = v;
    }
  return m;
}

/* Computes, for one position, the exit wave, its far field, the error terms
 * and Delta = F^-1(proj(F psi)) - psi, using probe Pc and the object as it
 * is.  Writes Delta (K values) and the pre-step patch O_old (K values). */
static void epie_delta(const cplx *O, int W, const cplx *Pc, int N, const double *I,
                       int y0, int x0, cplx *delta, cplx *Oold, double *err, double *isum) {
  const long K = (long)N * N;
  for (int y = 0; y < N; ++y)
    for (int x = 0; x < N; ++x) {
      long r = (long)y * N + x;
      Oold[r] = O[(long)(y0 + y) * W + x0 + x];
      delta[r] = Pc[r] * Oold[r]; /* psi */
    }
  cplx *Psi = (cplx *)malloc(sizeof(cplx) * K);
  memcpy(Psi, delta, sizeof(cplx) * K);
  orc_fft2(Psi, N, -1);
  orc_modulus_project(Psi, I, K, err, isum);
  orc_fft2(Psi, N, +1);
  for (long r = 0; r < K; ++r) delta[r] = Psi[r] - delta[r];
  free(Psi);
}

/* Sequential ePIE step at one position (in place on O and P).
 * O: H x W, P: N x N, I: N x N in FFT order, (y0, x0): patch top-left.
 * Returns 0, or -2 when the patch is not inside the object. */
int orc_epie_step(cplx *O, int H, int W, cplx *P, int N, const double *I,
                  int y0, int x0, double alpha, double beta, int omax_global,
                  double *err, double *isum) {
  if (y0 < 0 || x0 < 0 || y0 + N > H || x0 + N > W) return -2;
  const long K = (long)N * N;
  cplx *delta = (cplx *)malloc(sizeof(cplx) * K);
  cplx *Oold = (cplx *)malloc(sizeof(cplx) * K);
  double pmax = max_abs2(P, K);
  double omax = omax_global ? max_abs2(O, (long)H * W) : max_abs2_patch(O, W, y0, x0, N);
  epie_delta(O, W, P, N, I, y0, x0, delta, Oold, err, isum);
  double ao = pmax > 0.0 ? alpha / pmax : 0.0;
  double bp = omax > 0.0 ? beta / omax : 0.0;
  for (int y = 0; y < N; ++y)
    for (int x = 0; x < N; ++x) {
      long r = (long)y * N + x;
      cplx Pold = P[r];
      O[(long)(y0 + y) * W + x0 + x] = Oold[r] + ao * conj(Pold) * delta[r];
      P[r] = Pold + bp * conj(Oold[r]) * delta[r];
    }
  free(delta);
  free(Oold);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Sweeps over groups (sequential = groups of one; coloured = colour classes)*/
/* ------------------------------------------------------------------------ */

/* Runs the groups in the given order.  Members of a group all use the
 * probe Pc at group start; each updates its own object patch with Pc and
 * contributes beta conj(O_old)/max|O_old|^2 Delta to the probe move, which
 * is divided by the group size when probe_mean != 0 (R6).  Members of a
 * group with more than one member must have non-overlapping patches; this
 * is checked (-3).  I_all: frames x N*N FFT-order intensities indexed by
 * frame id; pos: frames x (y, x).  err/isum accumulate the error terms. */
int orc_sweep_groups(cplx *O, int H, int W, cplx *P, int N, const double *I_all,
                     const int32_t *pos, const int32_t *order, const int32_t *group_start,
                     int32_t n_groups, double alpha, double beta, int omax_global,
                     int probe_mean, double *err, double *isum) {
  const long K = (long)N * N;
  cplx *Pc = (cplx *)malloc(sizeof(cplx) * K);
  cplx *acc = (cplx *)malloc(sizeof(cplx) * K);
  cplx *delta = (cplx *)malloc(sizeof(cplx) * K);
  cplx *Oold = (cplx *)malloc(sizeof(cplx) * K);
  int rc = 0;
  for (int g = 0; g < n_groups && rc == 0; ++g) {
    int a = group_start[g], b = group_start[g + 1];
    for (int m = a; m < b && rc == 0; ++m) {
      int j = order[m], y0 = pos[2 * j], x0 = pos[2 * j + 1];
      if (y0 < 0 || x0 < 0 || y0 + N > H || x0 + N > W) rc = -2;
      for (int q = a; q < m && rc == 0; ++q) {
        int i = order[q];
        if (abs(pos[2 * i] - y0) < N && abs(pos[2 * i + 1] - x0) < N) rc = -3;
      }
    }
    if (rc) break;
    memcpy(Pc, P, sizeof(cplx) * K);
    memset(acc, 0, sizeof(cplx) * K);
    double pmax = max_abs2(Pc, K);
    double ao = pmax > 0.0 ? alpha / pmax : 0.0;
    double oglob = omax_global ? max_abs2(O, (long)H * W) : 0.0;
    for (int m = a; m < b; ++m) {
      int j = order[m], y0 = pos[2 * j], x0 = pos[2 * j + 1];
      double omax = omax_global ? oglob : max_abs2_patch(O, W, y0, x0, N);
      double bp = omax > 0.0 ? beta / omax : 0.0;
      epie_delta(O, W, Pc, N, I_all + (long)j * K, y0, x0, delta, Oold, err, isum);
      for (int y = 0; y < N; ++y)
        for (int x = 0; x < N; ++x) {
          long r = (long)y * N + x;
          O[(long)(y0 + y) * W + x0 + x] = Oold[r] + ao * conj(Pc[r]) * delta[r];
          acc[r] += bp * conj(Oold[r]) * delta[r];
        }
    }
    double scale = probe_mean ? 1.0 / (double)(b - a) : 1.0;
    for (long r = 0; r < K; ++r) P[r] = Pc[r] + scale * acc[r];
  }
  free(Pc);
  free(acc);
  free(delta);
  free(Oold);
  return rc;
}

/* Mini-batch sweep (R7): consecutive batches of `batch` positions of
 * `order` (n positions) share the batch-start O and P.
 * O(r) += alpha * sum_j [conj(P) Delta_j / max|P|^2](r) / max(1, cnt(r)),
 * P += (1/|batch|) * sum_j beta conj(O_j,old) Delta_j / max|O_j,old|^2. */
int orc_sweep_minibatch(cplx *O, int H, int W, cplx *P, int N, const double *I_all,
                        const int32_t *pos, const int32_t *order, int32_t n, int32_t batch,
                        double alpha, double beta, int omax_global, double *err,
                        double *isum) {
  if (batch < 1) return -1;
  const long K = (long)N * N, HW = (long)H * W;
  cplx *Pb = (cplx *)malloc(sizeof(cplx) * K);
  cplx *accP = (cplx *)malloc(sizeof(cplx) * K);
  cplx *accO = (cplx *)malloc(sizeof(cplx) * HW);
  int32_t *cnt = (int32_t *)malloc(sizeof(int32_t) * HW);
  cplx *delta = (cplx *)malloc(sizeof(cplx) * K);
  cplx *Oold = (cplx *)malloc(sizeof(cplx) * K);
  int rc = 0;
  for (int a = 0; a < n && rc == 0; a += batch) {
    int b = a + batch < n ? a + batch : n;
    for (int m = a; m < b; ++m) {
      int j = order[m], y0 = pos[2 * j], x0 = pos[2 * j + 1];
      if (y0 < 0 || x0 < 0 || y0 + N > H || x0 + N > W) rc = -2;
    }
    if (rc) break;
    memcpy(Pb, P, sizeof(cplx) * K);
    memset(accP, 0, sizeof(cplx) * K);
    memset(accO, 0, sizeof(cplx) * HW);
    memset(cnt, 0, sizeof(int32_t) * HW);
    double pmax = max_abs2(Pb, K);
    double ao = pmax > 0.0 ? 1.0 / pmax : 0.0;
    double oglob = omax_global ? max_abs2(O, HW) : 0.0;
    for (int m = a; m < b; ++m) {
      int j = order[m], y0 = pos[2 * j], x0 = pos[2 * j + 1];
      double omax = omax_global ? oglob : max_abs2_patch(O, W, y0, x0, N);
      double bp = omax > 0.0 ? beta / omax : 0.0;
      /* O is untouched inside the batch, so the batch-start state is read */
      epie_delta(O, W, Pb, N, I_all + (long)j * K, y0, x0, delta, Oold, err, isum);
      for (int y = 0; y < N; ++y)
        for (int x = 0; x < N; ++x) {
          long r = (long)y * N + x, o = (long)(y0 + y) * W + x0 + x;
          accO[o] += ao * conj(Pb[r]) * delta[r];
          cnt[o] += 1;
          accP[r] += bp * conj(Oold[r]) * delta[r];
        }
    }
    for (long o = 0; o < HW; ++o)
      if (cnt[o] > 0) O[o] += alpha * accO[o] / (double)cnt[o];
    for (long r = 0; r < K; ++r) P[r] = Pb[r] + accP[r] / (double)(b - a);
  }
  free(Pb);
  free(accP);
  free(accO);
  free(cnt);
  free(delta);
  free(Oold);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Visiting order and colour classes (R6, R9)                                */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood 2014; public-domain reference by Vigna). */
uint64_t orc_splitmix64(uint64_t *state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static uint64_t sweep_state(uint64_t seed, int64_t sweep) {
  return seed ^ ((uint64_t)sweep * 0xD1B54A32D192ED03ULL);
}

static void fisher_yates(int32_t *a, int32_t n, uint64_t *st) {
  for (int32_t i = n - 1; i >= 1; --i) {
    int32_t j = (int32_t)(orc_splitmix64(st) % (uint64_t)(i + 1));
    int32_t t = a[i];
    a[i] = a[j];
    a[j] = t;
  }
}

/* Sequential order of sweep `sweep`: a shuffled permutation of 0..n-1. */
void orc_order_sequential(uint64_t seed, int64_t sweep, int32_t n, int32_t *order) {
  uint64_t st = sweep_state(seed, sweep);
  for (int32_t i = 0; i < n; ++i) order[i] = i;
  fisher_yates(order, n, &st);
}

/* Greedy first-fit colouring in index (append) order: frames i and j
 * conflict iff |y_i - y_j| < N and |x_i - x_j| < N; each frame takes the
 * smallest class id that no earlier conflicting frame holds and that holds
 * fewer than `cap` frames (cap <= 0: no limit).  Returns the number of
 * classes. */
int32_t orc_colour_greedy(const int32_t *pos, int32_t n, int32_t N, int32_t cap, int32_t *colour) {
  int32_t ncls = 0;
  uint8_t *used = (uint8_t *)calloc((size_t)n + 1, 1);
  int32_t *size = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
  for (int32_t i = 0; i < n; ++i) {
    memset(used, 0, (size_t)ncls + 1);
    for (int32_t j = 0; j < i; ++j)
      if (abs(pos[2 * i] - pos[2 * j]) < N && abs(pos[2 * i + 1] - pos[2 * j + 1]) < N)
        used[colour[j]] = 1;
    int32_t c = 0;
    while (c < ncls && (used[c] || (cap > 0 && size[c] >= cap))) ++c;
    colour[i] = c;
    size[c] += 1;
    if (c == ncls) ++ncls;
  }
  free(used);
  free(size);
  return ncls;
}

/* Coloured order of sweep `sweep`: classes visited in a shuffled order
 * (Fisher-Yates over 0..ncls-1), then the members of each visited class
 * (listed in frame-index order) shuffled with the same continuing stream.
 * order: n frame ids; group_start: ncls+1 offsets into order. */
void orc_order_coloured(uint64_t seed, int64_t sweep, int32_t n, const int32_t *colour,
                        int32_t ncls, int32_t *order, int32_t *group_start) {
  uint64_t st = sweep_state(seed, sweep);
  int32_t *cls = (int32_t *)malloc(sizeof(int32_t) * (ncls > 0 ? ncls : 1));
  for (int32_t c = 0; c < ncls; ++c) cls[c] = c;
  fisher_yates(cls, ncls, &st);
  int32_t p = 0;
  for (int32_t g = 0; g < ncls; ++g) {
    group_start[g] = p;
    int32_t a = p;
    for (int32_t i = 0; i < n; ++i)
      if (colour[i] == cls[g]) order[p++] = i;
    fisher_yates(order + a, p - a, &st);
  }
  group_start[ncls] = p;
  free(cls);
}

/* ------------------------------------------------------------------------ */
/* Amplitude loss and its gradient (differentiable reconstruction)           */
/* ------------------------------------------------------------------------ */

/* L = sum_j sum_k (|F(S_dj P . O_j)|(k) - sqrt(I_j(k)))^2 with integer patch
 * offsets pos_j, sub-pixel shifts d_j = (dy, dx) applied to the probe as a
 * Fourier shift S_d P = F^-1[ F P . exp(-2 pi i (ky dy + kx dx)/N) ], with
 * k in FFT frequency order (k >= N/2 stands for k - N).  Gradients use the
 * convention dL/dRe + i dL/dIm for complex variables (gO: H x W,
 * gP: N x N) and dL/d(dy), dL/d(dx) for the shifts (gd: n x 2).
 * Where |Psi| = 0 the amplitude's gradient is taken as 0.  Returns L. */
double orc_amp_loss_grad(const cplx *O, int H, int W, const cplx *P, int N,
                         const double *I_all, const int32_t *pos, const double *shift,
                         int32_t n, cplx *gO, cplx *gP, double *gd) {
  const long K = (long)N * N;
  cplx *FP = (cplx *)malloc(sizeof(cplx) * K);
  cplx *Ps = (cplx *)malloc(sizeof(cplx) * K);
  cplx *Psi = (cplx *)malloc(sizeof(cplx) * K);
  cplx *G = (cplx *)malloc(sizeof(cplx) * K);
  cplx *gPs = (cplx *)malloc(sizeof(cplx) * K);
  if (gO) memset(gO, 0, sizeof(cplx) * (long)H * W);
  if (gP) memset(gP, 0, sizeof(cplx) * K);
  memcpy(FP, P, sizeof(cplx) * K);
  orc_fft2(FP, N, -1);
  double L = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    int y0 = pos[2 * j], x0 = pos[2 * j + 1];
    double dy = shift ? shift[2 * j] : 0.0, dx = shift ? shift[2 * j + 1] : 0.0;
    /* shifted probe */
    for (int ky = 0; ky < N; ++ky)
      for (int kx = 0; kx < N; ++kx) {
        double fy = ky < N / 2 ? ky : ky - N, fx = kx < N / 2 ? kx : kx - N;
        double ang = -2.0 * ORC_PI * (fy * dy + fx * dx) / (double)N;
        Ps[(long)ky * N + kx] = FP[(long)ky * N + kx] * mkc(cos(ang), sin(ang));
      }
    orc_fft2(Ps, N, +1);
    for (int y = 0; y < N; ++y)
      for (int x = 0; x < N; ++x)
        Psi[(long)y * N + x] = Ps[(long)y * N + x] * O[(long)(y0 + y) * W + x0 + x];
    orc_fft2(Psi, N, -1);
    const double *I = I_all + (long)j * K;
    /* dL/dPsi* direction: G = 2 (|Psi| - sqrt I) Psi/|Psi|  (conv. dRe + i dIm) */
    for (long k = 0; k < K; ++k) {
      double a = cabs(Psi[k]);
      double r = sqrt(I[k] > 0.0 ? I[k] : 0.0);
      L += (a - r) * (a - r);
      G[k] = a > 0.0 ? 2.0 * (a - r) * Psi[k] / a : 0.0;
    }
    /* back through F: grad wrt psi = F^H G = K * F^-1 G */
    orc_fft2(G, N, +1);
    for (long k = 0; k < K; ++k) G[k] *= (double)K;
    /* psi = Ps . O_j:  g_O = conj(Ps) g_psi,  g_Ps = conj(O_j) g_psi */
    for (int y = 0; y < N; ++y)
      for (int x = 0; x < N; ++x) {
        long r = (long)y * N + x, o = (long)(y0 + y) * W + x0 + x;
        if (gO) gO[o] += conj(Ps[r]) * G[r];
        gPs[r] = conj(O[o]) * G[r];
      }
    /* Ps = F^-1 (FP . ph):  g_FPph = (1/K) F g_Ps ; then the shift phase */
    orc_fft2(gPs, N, -1);
    for (long k = 0; k < K; ++k) gPs[k] /= (double)K;
    double gdy = 0.0, gdx = 0.0;
    for (int ky = 0; ky < N; ++ky)
      for (int kx = 0; kx < N; ++kx) {
        long k = (long)ky * N + kx;
        double fy = ky < N / 2 ? ky : ky - N, fx = kx < N / 2 ? kx : kx - N;
        double ang = -2.0 * ORC_PI * (fy * dy + fx * dx) / (double)N;
        cplx ph = mkc(cos(ang), sin(ang));
        cplx z = FP[k] * ph;          /* value that the shift produced */
        cplx gz = gPs[k];             /* dL/dz (conv.) */
        /* dz/d(dy) = z * (-2 pi i fy / N); dL/d(dy) = Re(conj(gz) dz/d(dy)) */
        cplx dzy = z * mkc(0.0, -2.0 * ORC_PI * fy / (double)N);
        cplx dzx = z * mkc(0.0, -2.0 * ORC_PI * fx / (double)N);
        gdy += creal(conj(gz) * dzy);
        gdx += creal(conj(gz) * dzx);
        gPs[k] = gz * conj(ph);       /* back to FP */
      }
    if (gd) {
      gd[2 * j] = gdy;
      gd[2 * j + 1] = gdx;
    }
    /* FP = F P: g_P = K F^-1 g_FP */
    orc_fft2(gPs, N, +1);
    if (gP)
      for (long k = 0; k < K; ++k) gP[k] += (double)K * gPs[k];
  }
  free(FP);
  free(Ps);
  free(Psi);
  free(G);
  free(gPs);
  return L;
}
