/*
 * refine_oracle.c — FP64 oracle of the refinement objective and its gradient.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.c).  Not in the paper: a continuous
 * refinement of a grid detection of the synthetic-tracking search (Sec. 2.1)
 * by maximising a Gaussian matched-filter log-likelihood over the motion and
 * position.  Definitions (the library's reading):
 *
 *   cutout    output pixels p = (cx - 32 + u, cy - 32 + w), u, w in [0, 64)
 *   S(p)      = sum_i B_i(p_x + vx dt_i, p_y + vy dt_i), dt_i = t_i - t_ref,
 *               B_i the bilinear interpolation of frame i with zero outside
 *               (taps at floor(X), floor(X)+1; weights 1-f, f)
 *   g(p)      = exp(-((p_x - x0)^2 + (p_y - y0)^2) / (2 s^2)),
 *               s = FWHM / (2 sqrt(2 ln 2))
 *   J         = F <g, S> - F^2 N <g, g> / 2          (N = number of frames)
 *   SNR       = <g, S> / sqrt(N <g, g>)
 *   dJ/dF     = <g, S> - F N <g, g>
 *   dJ/dx0    = F <dg/dx0, S> - F^2 N <g, dg/dx0>,  dg/dx0 = g (p_x - x0) / s^2
 *   dJ/dvx    = F sum_p g(p) sum_i dt_i dB_i/dX,     dB/dX the slope of the
 *               cell [floor X, floor X + 1] (right derivative at integers)
 *   (y0, vy likewise).
 * Pinned by tests/test_refine_oracle.py: closed forms for a noiseless mover
 * (F_hat = A, zero position gradient at the truth), a linear ramp (exact
 * velocity derivative), and central finite differences away from kinks.
 */
#include <math.h>
#include <stdint.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static double px(const float* fr, int W, int H, int64_t u, int64_t v) {
  if (u < 0 || v < 0 || u >= W || v >= H) return 0.0;
  return (double)fr[v * (int64_t)W + u];
}

/* theta: [n][5] (vx, vy, x0, y0, F); centre: [n][2] int (cx, cy).
 * Outputs J[n], snr[n], grad[n][5] (grad may be NULL). */
int oracle_refine_eval(const float* frames, int N, int H, int W, const double* t, double t_ref,
                       const double* theta, const int32_t* centre, int64_t n, double fwhm,
                       double* J, double* snr, double* grad) {
  const double s = fwhm / (2.0 * sqrt(2.0 * log(2.0)));
  const double inv2s2 = 1.0 / (2.0 * s * s);
  const int64_t P = (int64_t)W * H;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < n; ++c) {
    const double vx = theta[5 * c], vy = theta[5 * c + 1];
    const double x0 = theta[5 * c + 2], y0 = theta[5 * c + 3], F = theta[5 * c + 4];
    const int cx = centre[2 * c], cy = centre[2 * c + 1];
    double gS = 0, gg = 0, gxS = 0, gyS = 0, ggx = 0, ggy = 0, dvx = 0, dvy = 0;
    for (int w = 0; w < 64; ++w)
      for (int u = 0; u < 64; ++u) {
        const double pxx = cx - 32 + u, pyy = cy - 32 + w;
        const double ddx = pxx - x0, ddy = pyy - y0;
        const double g = exp(-(ddx * ddx + ddy * ddy) * inv2s2);
        const double gx = g * ddx / (s * s), gy = g * ddy / (s * s);
        double S = 0, dSx = 0, dSy = 0;
        for (int i = 0; i < N; ++i) {
          const double dt = t[i] - t_ref;
          const double X = pxx + vx * dt, Y = pyy + vy * dt;
          const double fxl = floor(X), fyl = floor(Y);
          const double fx = X - fxl, fy = Y - fyl;
          const int64_t uu = (int64_t)fxl, vv = (int64_t)fyl;
          const float* fr = frames + (int64_t)i * P;
          const double i00 = px(fr, W, H, uu, vv), i10 = px(fr, W, H, uu + 1, vv);
          const double i01 = px(fr, W, H, uu, vv + 1), i11 = px(fr, W, H, uu + 1, vv + 1);
          S += (1 - fy) * ((1 - fx) * i00 + fx * i10) + fy * ((1 - fx) * i01 + fx * i11);
          dSx += dt * ((1 - fy) * (i10 - i00) + fy * (i11 - i01));
          dSy += dt * ((1 - fx) * (i01 - i00) + fx * (i11 - i10));
        }
        gS += g * S;
        gg += g * g;
        gxS += gx * S;
        gyS += gy * S;
        ggx += g * gx;
        ggy += g * gy;
        dvx += g * dSx;
        dvy += g * dSy;
      }
    J[c] = F * gS - 0.5 * F * F * N * gg;
    snr[c] = gg > 0 ? gS / sqrt(N * gg) : 0.0;
    if (grad) {
      grad[5 * c] = F * dvx;
      grad[5 * c + 1] = F * dvy;
      grad[5 * c + 2] = F * gxS - F * F * N * ggx;
      grad[5 * c + 3] = F * gyS - F * F * N * ggy;
      grad[5 * c + 4] = gS - F * N * gg;
    }
  }
  return 0;
}
