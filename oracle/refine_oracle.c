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
 * The Gauss-Newton curvature below is pinned there too: it equals the
 * finite-difference Hessian of J at a zero-residual fit (position and flux),
 * the motion-position coupling of the bilinear stack within 15 %, and damped
 * steps reach a noiseless mover's parameters.
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

/* Gauss-Newton curvature of the refinement objective (the optimiser the
 * library reserves as optimizer 1).  Reading: up to a constant that does not
 * depend on theta, J is the log-likelihood of the frames under the model
 *   m_i(q) = F g(q - (x0, y0) - v dt_i)      (unit noise per frame pixel),
 * sampled on the cutout in reference coordinates, so Gauss-Newton replaces
 * -Hessian(J) by the model's J^T J summed over frames and cutout pixels:
 *   dm_i/dx0 = F Gx,  dm_i/dvx = dt_i F Gx,  dm_i/dF = g,
 *   Gx = dg/dx0 = g (p_x - x0) / s^2   (y likewise).
 * With T1 = sum_i dt_i and T2 = sum_i dt_i^2 the entries are
 *   [vx,vx] F^2 T2 <Gx,Gx>   [vx,vy] F^2 T2 <Gx,Gy>   [vy,vy] F^2 T2 <Gy,Gy>
 *   [vx,x0] F^2 T1 <Gx,Gx>   [vx,y0] F^2 T1 <Gx,Gy>   [vy,x0] F^2 T1 <Gx,Gy>
 *   [vy,y0] F^2 T1 <Gy,Gy>   [x0,x0] F^2 N <Gx,Gx>    [x0,y0] F^2 N <Gx,Gy>
 *   [y0,y0] F^2 N <Gy,Gy>    [vx,F] F T1 <g,Gx>       [vy,F] F T1 <g,Gy>
 *   [x0,F] F N <g,Gx>        [y0,F] F N <g,Gy>        [F,F] N <g,g>.
 * theta [n][5], centre [n][2] as above; H [n][5][5] in the order (vx, vy,
 * x0, y0, F), symmetric.  The frames do not enter. */
int oracle_refine_gn_matrix(int N, const double* t, double t_ref, const double* theta,
                            const int32_t* centre, int64_t n, double fwhm, double* H) {
  const double s = fwhm / (2.0 * sqrt(2.0 * log(2.0)));
  const double inv2s2 = 1.0 / (2.0 * s * s);
  double T1 = 0.0, T2 = 0.0;
  for (int i = 0; i < N; ++i) {
    const double dt = t[i] - t_ref;
    T1 += dt;
    T2 += dt * dt;
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < n; ++c) {
    const double x0 = theta[5 * c + 2], y0 = theta[5 * c + 3], F = theta[5 * c + 4];
    const int cx = centre[2 * c], cy = centre[2 * c + 1];
    double gg = 0, xx = 0, yy = 0, xy = 0, gx_ = 0, gy_ = 0;
    for (int w = 0; w < 64; ++w)
      for (int u = 0; u < 64; ++u) {
        const double ddx = (double)(cx - 32 + u) - x0, ddy = (double)(cy - 32 + w) - y0;
        const double g = exp(-(ddx * ddx + ddy * ddy) * inv2s2);
        const double Gx = g * ddx / (s * s), Gy = g * ddy / (s * s);
        gg += g * g;
        xx += Gx * Gx;
        yy += Gy * Gy;
        xy += Gx * Gy;
        gx_ += g * Gx;
        gy_ += g * Gy;
      }
    const double F2 = F * F;
    double* h = H + 25 * c;
    const double e[5][5] = {
        {F2 * T2 * xx, F2 * T2 * xy, F2 * T1 * xx, F2 * T1 * xy, F * T1 * gx_},
        {F2 * T2 * xy, F2 * T2 * yy, F2 * T1 * xy, F2 * T1 * yy, F * T1 * gy_},
        {F2 * T1 * xx, F2 * T1 * xy, F2 * N * xx, F2 * N * xy, F * N * gx_},
        {F2 * T1 * xy, F2 * T1 * yy, F2 * N * xy, F2 * N * yy, F * N * gy_},
        {F * T1 * gx_, F * T1 * gy_, F * N * gx_, F * N * gy_, N * gg}};
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b) h[5 * a + b] = e[a][b];
  }
  return 0;
}
