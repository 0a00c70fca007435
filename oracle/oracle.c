/*
 * oracle.c — plain, slow CPU oracle of the synthetic-tracking search.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library: every quantity is
 * recomputed here from its definition.
 *
 * What it computes (Burdanov, Hasler & de Wit 2023):
 *   Sec. 1    shift-and-stack: each frame is shifted along a predicted linear
 *             motion and the shifted frames are combined (summed); synthetic
 *             tracking repeats this over a grid of trial motions.
 *   Sec. 2.1  motion is linear with no constraint on position angle (a full
 *             2-D velocity grid); the output is a set of detections with
 *             pixel coordinates, motion and S/N; a detection needs the object
 *             in at least half of the images (the coverage rule).
 *   Sec. 2.1  (frame QC) per-frame sky level and sky standard deviation: the
 *             robust statistics used to normalise the frames.
 * The readings taken where the paper is silent (shift sign, rounding,
 * boundaries, SNR, tie rule, clipping) are stated at each function.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared.  -ffp-contract=off
 * is part of the definition: every product below is rounded before the sum.
 * Parity status: every function here is pinned by the tests named in its
 * comment; none is "parity unpinned" except where stated.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* a1: time offsets and shifts (Sec. 2.1 linear motion)                */
/* ------------------------------------------------------------------ */

/* Shift of one frame for one grid velocity.
 * Reading: the stack lives in reference-epoch coordinates, so frame i is
 * sampled at p + v*dt_i with dt_i = t_i - t_ref.  Nearest mode rounds half
 * up: floor(v*dt + 0.5).  Bilinear mode returns floor(v*dt) and the fraction.
 * v = v0 + a*dv is one FP64 multiply and one add (no contraction). */
static void shift_of(double v0, double dv, int a, double dt, int mode,
                     int64_t* s_int, double* frac) {
  double v = v0 + (double)a * dv;
  double s = v * dt;
  if (mode == 0) {
    *s_int = (int64_t)floor(s + 0.5);
    *frac = 0.0;
  } else {
    double fl = floor(s);
    *s_int = (int64_t)fl;
    *frac = s - fl;
  }
}

/* Shift table [N][nv]. Pinned by test_oracle_pins.py::test_shift_* (hand cases). */
int oracle_shift_tables(const double* t, int N, double t_ref, double v0, double dv,
                        int nv, int mode, int32_t* s_out, double* f_out) {
  for (int i = 0; i < N; ++i) {
    double dt = t[i] - t_ref;
    for (int a = 0; a < nv; ++a) {
      int64_t s;
      double f;
      shift_of(v0, dv, a, dt, mode, &s, &f);
      s_out[(int64_t)i * nv + a] = (int32_t)s;
      if (f_out) f_out[(int64_t)i * nv + a] = f;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* a2: robust sky statistics and normalisation (Sec. 2.1 frame QC)     */
/* ------------------------------------------------------------------ */

/* kappa-sigma clipped mean and population standard deviation of the finite
 * pixels of one frame, FP64.  Reading: start from all finite pixels; compute
 * mean and std of the kept set; keep |x - mean| <= kappa*std; stop when the
 * kept set does not change or after max_iter statistics.  Pinned by
 * test_oracle_pins.py::test_sky_stats_* (closed forms, hand-built outliers). */
int oracle_sky_stats(const float* x, int64_t n, double kappa, int max_iter,
                     double* mu_out, double* sigma_out, int64_t* kept_out,
                     int* iters_out) {
  unsigned char* keep = (unsigned char*)malloc((size_t)n);
  if (!keep) return -1;
  for (int64_t j = 0; j < n; ++j) keep[j] = isfinite(x[j]) ? 1 : 0;
  double mu = 0.0, sigma = 0.0;
  int64_t cnt = 0;
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    double sum = 0.0;
    cnt = 0;
    for (int64_t j = 0; j < n; ++j)
      if (keep[j]) { sum += (double)x[j]; ++cnt; }
    if (cnt == 0) { mu = 0.0; sigma = 0.0; break; }
    mu = sum / (double)cnt;
    double ss = 0.0;
    for (int64_t j = 0; j < n; ++j)
      if (keep[j]) { double d = (double)x[j] - mu; ss += d * d; }
    sigma = sqrt(ss / (double)cnt);
    if (it == max_iter) break;
    int64_t changed = 0;
    for (int64_t j = 0; j < n; ++j) {
      unsigned char k2 = 0;
      if (isfinite(x[j])) k2 = fabs((double)x[j] - mu) <= kappa * sigma ? 1 : 0;
      if (k2 != keep[j]) { ++changed; keep[j] = k2; }
    }
    if (changed == 0) break;
  }
  free(keep);
  *mu_out = mu;
  *sigma_out = sigma;
  if (kept_out) *kept_out = cnt;
  if (iters_out) *iters_out = it > max_iter ? max_iter : it;
  return 0;
}

/* I = (R - mu)/sigma rounded to FP32; NaN (and any non-finite) -> 0; with
 * cr_clip > 0, |I| > cr_clip -> 0.  A frame with sigma == 0 maps to 0. */
int oracle_normalize(const float* raw, int N, int64_t npix, double kappa, int max_iter,
                     float cr_clip, float* out, double* mu, double* sigma) {
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
  for (int i = 0; i < N; ++i) {
    const float* r = raw + (int64_t)i * npix;
    float* o = out + (int64_t)i * npix;
    double m, s;
    if (oracle_sky_stats(r, npix, kappa, max_iter, &m, &s, NULL, NULL) != 0) { err |= 1; continue; }
    mu[i] = m;
    sigma[i] = s;
    for (int64_t j = 0; j < npix; ++j) {
      float v = 0.0f;
      if (isfinite(r[j]) && s > 0.0) v = (float)(((double)r[j] - m) / s);
      if (cr_clip > 0.0f && fabsf(v) > cr_clip) v = 0.0f;
      o[j] = v;
    }
  }
  return err ? -1 : 0;
}

/* Round-to-nearest-even FP32 -> BF16 -> FP32, the value a BF16 frame store
 * holds.  NaN stays NaN. */
static float bf16_round(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) {
    u |= 0x00400000u;
  } else {
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
  }
  u &= 0xffff0000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

/* Values a BF16 store holds, for the FP32-sequential oracle over BF16 frames. */
int oracle_round_bf16(const float* in, int64_t n, float* out) {
  for (int64_t j = 0; j < n; ++j) out[j] = bf16_round(in[j]);
  return 0;
}

/* ------------------------------------------------------------------ */
/* a3/a4: shift-and-stack of one velocity plane (Sec. 1, Sec. 2.1)     */
/* ------------------------------------------------------------------ */

typedef struct {
  const float* frames;
  int N, H, W;
  const double* t;
  double t_ref, vx0, dvx, vy0, dvy;
  int nvx, nvy;
  int mode;  /* 0 nearest, 1 bilinear */
  int prec;  /* 0 FP64 accumulation, 1 FP32 sequential accumulation */
} problem;

static float pix(const problem* p, int i, int64_t x, int64_t y) {
  if (x < 0 || y < 0 || x >= p->W || y >= p->H) return 0.0f;
  return p->frames[((int64_t)i * p->H + y) * p->W + x];
}

/* S_k(x, y) and n_cov for one output, summing frames i = 0..N-1 in order. */
static void stack_point(const problem* p, int x, int y, int k, double* S, int32_t* C) {
  int a = k % p->nvx, b = k / p->nvx;
  double acc64 = 0.0;
  float acc32 = 0.0f;
  int32_t n = 0;
  for (int i = 0; i < p->N; ++i) {
    double dt = p->t[i] - p->t_ref;
    int64_t sx, sy;
    double fx, fy;
    shift_of(p->vx0, p->dvx, a, dt, p->mode, &sx, &fx);
    shift_of(p->vy0, p->dvy, b, dt, p->mode, &sy, &fy);
    int64_t u = x + sx, v = y + sy;
    if (p->mode == 0) {
      int inside = u >= 0 && u < p->W && v >= 0 && v < p->H;
      n += inside;
      float s = pix(p, i, u, v);
      acc64 += (double)s;
      acc32 = acc32 + s;
    } else {
      int inx = u >= 0 && (u <= p->W - 2 || (u == p->W - 1 && fx == 0.0));
      int iny = v >= 0 && (v <= p->H - 2 || (v == p->H - 1 && fy == 0.0));
      n += inx && iny;
      double s = (1.0 - fy) * ((1.0 - fx) * pix(p, i, u, v) + fx * pix(p, i, u + 1, v)) +
                 fy * ((1.0 - fx) * pix(p, i, u, v + 1) + fx * pix(p, i, u + 1, v + 1));
      acc64 += s;
      acc32 = acc32 + (float)s;
    }
  }
  *S = p->prec == 1 ? (double)acc32 : acc64;
  *C = n;
}

/* Whole plane k, accumulated frame by frame; same per-output order as
 * stack_point. */
static void stack_plane(const problem* p, int k, double* S, int32_t* C) {
  int64_t P = (int64_t)p->H * p->W;
  int a = k % p->nvx, b = k / p->nvx;
  float* S32 = NULL;
  if (p->prec == 1) S32 = (float*)calloc((size_t)P, sizeof(float));
  for (int64_t j = 0; j < P; ++j) { S[j] = 0.0; C[j] = 0; }
  for (int i = 0; i < p->N; ++i) {
    double dt = p->t[i] - p->t_ref;
    int64_t sx, sy;
    double fx, fy;
    shift_of(p->vx0, p->dvx, a, dt, p->mode, &sx, &fx);
    shift_of(p->vy0, p->dvy, b, dt, p->mode, &sy, &fy);
    for (int y = 0; y < p->H; ++y) {
      int64_t v = y + sy;
      for (int x = 0; x < p->W; ++x) {
        int64_t u = x + sx;
        int64_t j = (int64_t)y * p->W + x;
        if (p->mode == 0) {
          float s = pix(p, i, u, v);
          C[j] += (u >= 0 && u < p->W && v >= 0 && v < p->H);
          if (S32) S32[j] = S32[j] + s; else S[j] += (double)s;
        } else {
          int inx = u >= 0 && (u <= p->W - 2 || (u == p->W - 1 && fx == 0.0));
          int iny = v >= 0 && (v <= p->H - 2 || (v == p->H - 1 && fy == 0.0));
          C[j] += inx && iny;
          double s = (1.0 - fy) * ((1.0 - fx) * pix(p, i, u, v) + fx * pix(p, i, u + 1, v)) +
                     fy * ((1.0 - fx) * pix(p, i, u, v + 1) + fx * pix(p, i, u + 1, v + 1));
          if (S32) S32[j] = S32[j] + (float)s; else S[j] += s;
        }
      }
    }
  }
  if (S32) {
    for (int64_t j = 0; j < P; ++j) S[j] = (double)S32[j];
    free(S32);
  }
}

/* Planes for a list of velocity indices: S_out, C_out are [nk][H][W].
 * Pinned by test_oracle_pins.py: zero velocity == frame sum, noiseless
 * injection, linearity, time reversal, translation, bilinear ramp and
 * constant closed forms, integer-fraction reduction, pure-noise statistics. */
int oracle_stack_planes(const float* frames, int N, int H, int W, const double* t,
                        double t_ref, double vx0, double dvx, int nvx, double vy0,
                        double dvy, int nvy, int mode, int prec, const int32_t* klist,
                        int nk, double* S_out, int32_t* C_out) {
  problem p = {frames, N, H, W, t, t_ref, vx0, dvx, vy0, dvy, nvx, nvy, mode, prec};
  int64_t P = (int64_t)H * W;
#pragma omp parallel for schedule(dynamic, 1)
  for (int q = 0; q < nk; ++q) stack_plane(&p, klist[q], S_out + q * P, C_out + q * P);
  return 0;
}

/* Individual outputs (x, y, k) triples: for sampled parity at full size. */
int oracle_stack_points(const float* frames, int N, int H, int W, const double* t,
                        double t_ref, double vx0, double dvx, int nvx, double vy0,
                        double dvy, int nvy, int mode, int prec, const int32_t* xyk,
                        int64_t npts, double* S_out, int32_t* C_out) {
  problem p = {frames, N, H, W, t, t_ref, vx0, dvx, vy0, dvy, nvx, nvy, mode, prec};
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t q = 0; q < npts; ++q)
    stack_point(&p, xyk[3 * q], xyk[3 * q + 1], xyk[3 * q + 2], S_out + q, C_out + q);
  return 0;
}

/* ------------------------------------------------------------------ */
/* a5/a6: threshold, coverage rule, local maxima, sorted list          */
/* ------------------------------------------------------------------ */

typedef struct {
  int32_t x, y, k, n_cov;
  double stack, snr;
} oracle_cand;

/* Threshold thr[n] = (float)(tau*sqrt(n)) and 1/sqrt(n) as FP32, FP64 formulas. */
static float thr_of(float tau, int n) { return (float)((double)tau * sqrt((double)n)); }
static float rsq_of(int n) { return n > 0 ? (float)(1.0 / sqrt((double)n)) : 0.0f; }

/* Candidates of one plane in raster order.  Reading of Sec. 2.1: a detection
 * needs n_cov >= n_min (at least half of the images by default), S >= thr,
 * and S a local maximum over the 8 in-frame neighbours with n_cov >= n_min:
 * strictly greater than earlier neighbours (raster order), >= later ones. */
static int64_t plane_candidates(const problem* p, int k, const double* S, const int32_t* C,
                                float tau, int nmin, oracle_cand* out, int64_t cap) {
  int64_t n = 0;
  for (int y = 0; y < p->H; ++y)
    for (int x = 0; x < p->W; ++x) {
      int64_t j = (int64_t)y * p->W + x;
      int c = C[j];
      if (c < nmin) continue;
      double s = S[j];
      float th = thr_of(tau, c);
      if (p->prec == 1) {
        if (!((float)s >= th)) continue;
      } else {
        if (!(s >= (double)th)) continue;
      }
      int ok = 1;
      for (int dy = -1; dy <= 1 && ok; ++dy)
        for (int dx = -1; dx <= 1 && ok; ++dx) {
          if (!dx && !dy) continue;
          int qx = x + dx, qy = y + dy;
          if (qx < 0 || qy < 0 || qx >= p->W || qy >= p->H) continue;
          int64_t jq = (int64_t)qy * p->W + qx;
          if (C[jq] < nmin) continue;
          int earlier = dy < 0 || (dy == 0 && dx < 0);
          if (earlier ? !(s > S[jq]) : !(s >= S[jq])) ok = 0;
        }
      if (!ok) continue;
      if (n < cap && out) {
        out[n].x = x;
        out[n].y = y;
        out[n].k = k;
        out[n].n_cov = c;
        out[n].stack = s;
        out[n].snr = p->prec == 1 ? (double)((float)s * rsq_of(c)) : s / sqrt((double)c);
      }
      ++n;
    }
  return n;
}

/* Search over velocity indices [k_begin, k_end): candidates sorted by
 * (k, y, x).  Returns the total count (records beyond cap are not written),
 * or -1 on allocation failure.  nmin <= 0 selects ceil(N/2).  Pinned by
 * tests/golden/ hand-built tie, plateau, threshold-equality and coverage
 * fixtures and by the noiseless injection test. */
int64_t oracle_search(const float* frames, int N, int H, int W, const double* t,
                      double t_ref, double vx0, double dvx, int nvx, double vy0, double dvy,
                      int nvy, int mode, int prec, float tau, int nmin, int32_t k_begin,
                      int32_t k_end, oracle_cand* out, int64_t cap) {
  problem p = {frames, N, H, W, t, t_ref, vx0, dvx, vy0, dvy, nvx, nvy, mode, prec};
  if (nmin <= 0) nmin = (N + 1) / 2;
  int nk = k_end - k_begin;
  if (nk <= 0) return 0;
  int64_t P = (int64_t)H * W;
  int64_t* counts = (int64_t*)calloc((size_t)nk, sizeof(int64_t));
  oracle_cand** lists = (oracle_cand**)calloc((size_t)nk, sizeof(oracle_cand*));
  int fail = 0;
#pragma omp parallel reduction(| : fail)
  {
    double* S = (double*)malloc((size_t)P * sizeof(double));
    int32_t* C = (int32_t*)malloc((size_t)P * sizeof(int32_t));
    if (!S || !C) fail |= 1;
#pragma omp for schedule(dynamic, 1)
    for (int q = 0; q < nk; ++q) {
      if (!S || !C) continue;
      int k = k_begin + q;
      stack_plane(&p, k, S, C);
      int64_t c = plane_candidates(&p, k, S, C, tau, nmin, NULL, 0);
      counts[q] = c;
      if (c > 0) {
        lists[q] = (oracle_cand*)malloc((size_t)c * sizeof(oracle_cand));
        if (!lists[q]) { fail |= 1; continue; }
        plane_candidates(&p, k, S, C, tau, nmin, lists[q], c);
      }
    }
    free(S);
    free(C);
  }
  int64_t total = 0;
  for (int q = 0; q < nk; ++q) {
    for (int64_t j = 0; j < counts[q]; ++j) {
      if (out && total < cap && lists[q]) out[total] = lists[q][j];
      ++total;
    }
    free(lists[q]);
  }
  free(lists);
  free(counts);
  return fail ? -1 : total;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the following parallel regions (n >= 1); no effect without
 * OpenMP.  For a process that runs alone although its launcher limited each
 * process to one thread. */
void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
