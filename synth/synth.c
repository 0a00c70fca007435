/*
 * synth.c — seeded synthetic fields for the synthetic-tracking search.
 *
 * Generates the inputs only: Gaussian sky noise, a smoothed sky residual,
 * masked star blobs, cosmic-ray hits and Gaussian-PSF movers on linear
 * trajectories.  It contains none of the search's arithmetic (no stacking,
 * thresholding or statistics).  Random numbers come from the counter-based
 * Philox4x32-10 generator (Salmon, Moraes, Dror & Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), keyed by the seed and indexed by
 * (element, stream), so the output does not depend on thread count or order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static inline void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

/* Philox4x32 with 10 rounds: multipliers 0xD2511F53, 0xCD9E8D57; Weyl key
 * increments 0x9E3779B9, 0xBB67AE85 (the published constants). */
static void philox4x32_10(const uint32_t in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
    mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Raw Philox words: out[4*j .. 4*j+3] for counter j of the stream. */
void synth_philox(uint64_t seed, uint64_t stream, uint64_t first, int64_t n_blocks, uint32_t* out) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t j = 0; j < n_blocks; ++j) {
    uint64_t c = first + (uint64_t)j;
    uint32_t in[4] = {(uint32_t)c, (uint32_t)(c >> 32), (uint32_t)stream, (uint32_t)(stream >> 32)};
    philox4x32_10(in, key, out + 4 * j);
  }
}

/* n standard normals times sigma (Box-Muller on pairs of 32-bit uniforms in (0, 1]). */
void synth_normal(float* out, int64_t n, uint64_t seed, uint64_t stream, float sigma) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  int64_t nb = (n + 3) / 4;
  const double two_pi = 6.283185307179586476925286766559;
  const double inv32 = 1.0 / 4294967296.0;
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < nb; ++j) {
    uint32_t in[4] = {(uint32_t)j, (uint32_t)((uint64_t)j >> 32), (uint32_t)stream,
                      (uint32_t)(stream >> 32)};
    uint32_t r[4];
    philox4x32_10(in, key, r);
    float z[4];
    for (int h = 0; h < 2; ++h) {
      double u1 = ((double)r[2 * h] + 1.0) * inv32;
      double u2 = (double)r[2 * h + 1] * inv32;
      double rad = sqrt(-2.0 * log(u1));
      z[2 * h] = (float)(sigma * rad * cos(two_pi * u2));
      z[2 * h + 1] = (float)(sigma * rad * sin(two_pi * u2));
    }
    for (int q = 0; q < 4; ++q)
      if (4 * j + q < n) out[4 * j + q] = z[q];
  }
}

/* Adds sigma * (box mean of width 2r+1 of fresh unit normals) to each of the N
 * frames: a spatially correlated residual whose std is sigma/(2r+1) before the
 * caller's scaling.  Edges use the clipped window. */
void synth_add_smooth_residual(float* frames, int N, int H, int W, uint64_t seed, int r,
                               float scale) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < N; ++i) {
    float* buf = (float*)malloc((size_t)H * W * sizeof(float));
    double* row = (double*)malloc((size_t)(W > H ? W : H) * sizeof(double));
    float* tmp = (float*)malloc((size_t)H * W * sizeof(float));
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int64_t n = (int64_t)H * W;
    const double two_pi = 6.283185307179586476925286766559;
    const double inv32 = 1.0 / 4294967296.0;
    for (int64_t j = 0; j < (n + 3) / 4; ++j) {
      uint32_t in[4] = {(uint32_t)j, (uint32_t)((uint64_t)j >> 32), (uint32_t)(0x5000 + i), 0u};
      uint32_t rr[4];
      philox4x32_10(in, key, rr);
      for (int h = 0; h < 2; ++h) {
        double u1 = ((double)rr[2 * h] + 1.0) * inv32;
        double u2 = (double)rr[2 * h + 1] * inv32;
        double rad = sqrt(-2.0 * log(u1));
        if (4 * j + 2 * h < n) buf[4 * j + 2 * h] = (float)(rad * cos(two_pi * u2));
        if (4 * j + 2 * h + 1 < n) buf[4 * j + 2 * h + 1] = (float)(rad * sin(two_pi * u2));
      }
    }
    /* horizontal then vertical box mean */
    for (int y = 0; y < H; ++y) {
      double acc = 0.0;
      for (int x = 0; x < W; ++x) row[x] = buf[(int64_t)y * W + x];
      for (int x = 0; x < W; ++x) {
        acc = 0.0;
        int c = 0;
        for (int d = -r; d <= r; ++d)
          if (x + d >= 0 && x + d < W) { acc += row[x + d]; ++c; }
        tmp[(int64_t)y * W + x] = (float)(acc / c);
      }
    }
    for (int x = 0; x < W; ++x) {
      for (int y = 0; y < H; ++y) row[y] = tmp[(int64_t)y * W + x];
      for (int y = 0; y < H; ++y) {
        double acc = 0.0;
        int c = 0;
        for (int d = -r; d <= r; ++d)
          if (y + d >= 0 && y + d < H) { acc += row[y + d]; ++c; }
        frames[(int64_t)i * n + (int64_t)y * W + x] += (float)(scale * acc / c);
      }
    }
    free(buf);
    free(row);
    free(tmp);
  }
}

/* Point-sampled Gaussian PSFs of movers on linear trajectories:
 * centre_i = (x0 + vx*(t_i - t_ref), y0 + vy*(t_i - t_ref)); peak amplitude
 * amp; sigma_psf = FWHM / (2 sqrt(2 ln 2)); rendered within 4 sigma.
 * movers: [M][5] = x0, y0, vx, vy, amp. */
void synth_render_movers(float* frames, int N, int H, int W, const double* t, double t_ref,
                         const double* movers, int M, double fwhm) {
  double sp = fwhm / (2.0 * sqrt(2.0 * log(2.0)));
  int rad = (int)ceil(4.0 * sp);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < N; ++i) {
    double dt = t[i] - t_ref;
    float* f = frames + (int64_t)i * H * W;
    for (int m = 0; m < M; ++m) {
      double cx = movers[5 * m] + movers[5 * m + 2] * dt;
      double cy = movers[5 * m + 1] + movers[5 * m + 3] * dt;
      double amp = movers[5 * m + 4];
      int ix = (int)floor(cx + 0.5), iy = (int)floor(cy + 0.5);
      for (int y = iy - rad; y <= iy + rad; ++y) {
        if (y < 0 || y >= H) continue;
        for (int x = ix - rad; x <= ix + rad; ++x) {
          if (x < 0 || x >= W) continue;
          double dx = x - cx, dy = y - cy;
          f[(int64_t)y * W + x] += (float)(amp * exp(-(dx * dx + dy * dy) / (2.0 * sp * sp)));
        }
      }
    }
  }
}

/* Single-pixel cosmic-ray hits: the number per frame is rate*H*W rounded,
 * positions uniform, amplitudes uniform in [amin, amax].  Returns the hits
 * written (<= cap) as [frame, x, y] triples in hits (may be NULL). */
int64_t synth_add_cosmics(float* frames, int N, int H, int W, uint64_t seed, double rate,
                          double amin, double amax, int32_t* hits, int64_t cap) {
  int64_t per = (int64_t)floor(rate * (double)H * (double)W + 0.5);
  int64_t total = 0;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int i = 0; i < N; ++i) {
    for (int64_t h = 0; h < per; ++h) {
      uint32_t in[4] = {(uint32_t)h, 0u, (uint32_t)(0x7000 + i), 1u};
      uint32_t r[4];
      philox4x32_10(in, key, r);
      int x = (int)((uint64_t)r[0] * (uint64_t)W >> 32);
      int y = (int)((uint64_t)r[1] * (uint64_t)H >> 32);
      double u = (double)r[2] / 4294967296.0;
      frames[((int64_t)i * H + y) * W + x] += (float)(amin + (amax - amin) * u);
      if (hits && total < cap) {
        hits[3 * total] = i;
        hits[3 * total + 1] = x;
        hits[3 * total + 2] = y;
      }
      ++total;
    }
  }
  return total;
}

/* Fixed-star residual blobs masked to NaN in every frame: pixels within
 * radius r of (x, y).  blobs: [B][3] = x, y, r. */
void synth_mask_blobs(float* frames, int N, int H, int W, const double* blobs, int B) {
  int64_t P = (int64_t)H * W;
  unsigned char* mask = (unsigned char*)calloc((size_t)P, 1);
  for (int b = 0; b < B; ++b) {
    double cx = blobs[3 * b], cy = blobs[3 * b + 1], r = blobs[3 * b + 2];
    int x0 = (int)floor(cx - r), x1 = (int)ceil(cx + r);
    int y0 = (int)floor(cy - r), y1 = (int)ceil(cy + r);
    for (int y = y0; y <= y1; ++y)
      for (int x = x0; x <= x1; ++x) {
        if (x < 0 || y < 0 || x >= W || y >= H) continue;
        double dx = x - cx, dy = y - cy;
        if (dx * dx + dy * dy <= r * r) mask[(int64_t)y * W + x] = 1;
      }
  }
  float nanv = NAN;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < N; ++i)
    for (int64_t j = 0; j < P; ++j)
      if (mask[j]) frames[(int64_t)i * P + j] = nanv;
  free(mask);
}
