// k_refine.cu — differentiable refinement of candidates (forward + adjoint).
//
// Not in the paper: a continuous refinement of the grid detections of the
// synthetic-tracking search (Sec. 2.1).  For theta = (vx, vy, x0, y0, F) and a
// 64 x 64 output cutout centred on the candidate pixel:
//   S(p)   = sum_i B_i(p + v dt_i)      bilinear stack, zero outside the frame
//   g(p)   = exp(-|p - (x0, y0)|^2 / (2 s^2)),  s = FWHM / (2 sqrt(2 ln 2))
//   J      = F <g, S> - F^2 N <g, g> / 2,  SNR = <g, S> / sqrt(N <g, g>)
// and the adjoint: dJ/dF = <g,S> - F N <g,g>; dJ/dx0 = F <dg/dx0, S> -
// F^2 N <g, dg/dx0>; dJ/dvx = F sum_p g(p) sum_i dt_i dB_i/dX (the slope of
// the bilinear cell).  The samples and their derivatives are recomputed on
// every evaluation, never stored.
//
// One CTA per candidate; thread t owns cutout row t/4 and 16 consecutive
// columns (t%4)*16.., so its pixels share one bilinear fraction per frame and
// their taps are contiguous.  Reductions use a fixed-order block tree.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "st_internal.h"
#include "st_sample.cuh"

namespace st {

namespace {

constexpr int kCut = 64;        // cutout side
constexpr int kThreads = 256;
constexpr int kPix = kCut * kCut / kThreads;  // 16 pixels per thread
constexpr int kSums = 8;

struct RefineArgs {
  const FieldDev* fds;          // device field descriptors
  const double* const* times;   // per field: device FP64 timestamps
  const double* t_ref;          // per field
  const float* theta_in;        // [n][5] (eval mode)
  const int32_t* centre_in;     // [n][2] (eval mode)
  const int32_t* field_in;      // [n]    (eval mode)
  const st_candidate* cand;     // [n]    (optimise mode)
  const double* grid;           // per field: vx0, dvx, vy0, dvy (optimise mode)
  int64_t n;
  float inv2s2, inv_s2;
  int steps;
  float lr_pos, lr_vel;
  float* J;
  float* snr;
  float* grad;                  // [n][5] or null
  st_refined* out;              // optimise mode
};

template <typename T>
__device__ __forceinline__ float pxv(const T* fr, int W, int H, int u, int v) {
  return (u >= 0 && v >= 0 && u < W && v < H) ? load_px<T>(fr + (int64_t)v * W + u) : 0.0f;
}

// Fixed-order block reduction of kSums values; result valid in thread 0.
__device__ void block_sum(float (&v)[kSums], float* sh) {
#pragma unroll
  for (int k = 0; k < kSums; ++k)
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], d);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < kSums; ++k) sh[warp * kSums + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < kSums; ++k) {
      float s = 0.0f;
      for (int w = 0; w < kThreads / 32; ++w) s += sh[w * kSums + k];
      v[k] = s;
    }
  __syncthreads();
}

// Sums for one candidate at theta: <g,S>, <g,g>, <gx,S>, <gy,S>, <g,gx>,
// <g,gy>, sum g dS/dvx, sum g dS/dvy (valid in thread 0).
template <typename T>
__device__ void evaluate(const FieldDev& fd, const double* t, double t_ref, int cx, int cy,
                         float vx, float vy, float x0, float y0, float inv2s2, float inv_s2,
                         float (&sums)[kSums], float* sh) {
  const int row = threadIdx.x / 4;
  const int col0 = (threadIdx.x % 4) * kPix;
  const float py = (float)(cy - kCut / 2 + row);
  const float px0 = (float)(cx - kCut / 2 + col0);
  float S[kPix];
  float g[kPix];
  const float dy0 = py - y0;
#pragma unroll
  for (int k = 0; k < kPix; ++k) {
    S[k] = 0.0f;
    const float dx = px0 + (float)k - x0;
    g[k] = expf(-(dx * dx + dy0 * dy0) * inv2s2);
  }
  float dvx = 0.0f, dvy = 0.0f;
  const T* cube = (const T*)fd.cube;
  const int64_t P = (int64_t)fd.W * fd.H;
  for (int i = 0; i < fd.N; ++i) {
    const float dt = (float)(t[i] - t_ref);
    const float X = px0 + vx * dt, Y = py + vy * dt;
    const float fxl = floorf(X), fyl = floorf(Y);
    const float fx = X - fxl, fy = Y - fyl;
    const int u = (int)fxl, v = (int)fyl;
    const T* fr = cube + (int64_t)i * P;
    float a0 = pxv<T>(fr, fd.W, fd.H, u, v), b0 = pxv<T>(fr, fd.W, fd.H, u, v + 1);
    float gdx = 0.0f, gdy = 0.0f;
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
      const float a1 = pxv<T>(fr, fd.W, fd.H, u + k + 1, v);
      const float b1 = pxv<T>(fr, fd.W, fd.H, u + k + 1, v + 1);
      const float top = a0 + fx * (a1 - a0), bot = b0 + fx * (b1 - b0);
      S[k] += top + fy * (bot - top);
      gdx += g[k] * ((1.0f - fy) * (a1 - a0) + fy * (b1 - b0));
      gdy += g[k] * (bot - top);
      a0 = a1;
      b0 = b1;
    }
    dvx += dt * gdx;
    dvy += dt * gdy;
  }
#pragma unroll
  for (int k = 0; k < kSums; ++k) sums[k] = 0.0f;
#pragma unroll
  for (int k = 0; k < kPix; ++k) {
    const float gx = g[k] * (px0 + (float)k - x0) * inv_s2;
    const float gy = g[k] * dy0 * inv_s2;
    sums[0] += g[k] * S[k];
    sums[1] += g[k] * g[k];
    sums[2] += gx * S[k];
    sums[3] += gy * S[k];
    sums[4] += g[k] * gx;
    sums[5] += g[k] * gy;
  }
  sums[6] = dvx;
  sums[7] = dvy;
  block_sum(sums, sh);
}

__device__ void objective(const float (&s)[kSums], int N, float F, float* J, float* snr,
                          float (&gr)[5]) {
  const float nf = (float)N;
  *J = F * s[0] - 0.5f * F * F * nf * s[1];
  *snr = s[1] > 0.0f ? s[0] / sqrtf(nf * s[1]) : 0.0f;
  gr[0] = F * s[6];
  gr[1] = F * s[7];
  gr[2] = F * s[2] - F * F * nf * s[4];
  gr[3] = F * s[3] - F * F * nf * s[5];
  gr[4] = s[0] - F * nf * s[1];
}

template <typename T, bool OPT>
__global__ void __launch_bounds__(kThreads) k_refine(RefineArgs a) {
  __shared__ float sh[(kThreads / 32) * kSums];
  __shared__ float th[5];
  const int64_t c = blockIdx.x;
  if (c >= a.n) return;
  int fi, cx, cy;
  if (OPT) {
    const st_candidate cd = a.cand[c];
    fi = cd.field;
    cx = cd.x;
    cy = cd.y;
  } else {
    fi = a.field_in[c];
    cx = a.centre_in[2 * c];
    cy = a.centre_in[2 * c + 1];
  }
  const FieldDev& fd = a.fds[fi];
  const double* t = a.times[fi];
  const double t_ref = a.t_ref[fi];
  if (threadIdx.x == 0) {
    if (OPT) {
      const st_candidate cd = a.cand[c];
      const double* gr = a.grid + 4 * fi;
      th[0] = (float)(gr[0] + (cd.k % fd.nvx) * gr[1]);
      th[1] = (float)(gr[2] + (cd.k / fd.nvx) * gr[3]);
      th[2] = (float)cd.x;
      th[3] = (float)cd.y;
      th[4] = 0.0f;
    } else {
      for (int k = 0; k < 5; ++k) th[k] = a.theta_in[5 * c + k];
    }
  }
  __syncthreads();
  float sums[kSums];
  float m[4] = {0, 0, 0, 0}, v2[4] = {0, 0, 0, 0};
  const int steps = OPT ? a.steps : 0;
  for (int step = 0; step <= steps; ++step) {
    evaluate<T>(fd, t, t_ref, cx, cy, th[0], th[1], th[2], th[3], a.inv2s2, a.inv_s2, sums, sh);
    if (threadIdx.x == 0) {
      // F at its optimum <g,S>/(N <g,g>) when optimising (profile likelihood)
      if (OPT) th[4] = sums[1] > 0.0f ? sums[0] / ((float)fd.N * sums[1]) : 0.0f;
      float J, snr, gr[5];
      objective(sums, fd.N, th[4], &J, &snr, gr);
      if (step == steps) {
        if (a.J) a.J[c] = J;
        if (a.snr) a.snr[c] = snr;
        if (a.grad)
          for (int k = 0; k < 5; ++k) a.grad[5 * c + k] = gr[k];
        if (OPT) {
          st_refined r;
          r.vx = th[0];
          r.vy = th[1];
          r.x0 = th[2];
          r.y0 = th[3];
          r.flux = th[4];
          r.snr = snr;
          r.obj = J;
          r.field = fi;
          a.out[c] = r;
        }
      } else {
        // Adam ascent on (vx, vy, x0, y0)
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.0f - __powf(b1, (float)(step + 1));
        const float c2 = 1.0f - __powf(b2, (float)(step + 1));
        for (int k = 0; k < 4; ++k) {
          m[k] = b1 * m[k] + (1.0f - b1) * gr[k];
          v2[k] = b2 * v2[k] + (1.0f - b2) * gr[k] * gr[k];
          const float lr = k < 2 ? a.lr_vel : a.lr_pos;
          th[k] += lr * (m[k] / c1) / (sqrtf(v2[k] / c2) + 1e-12f);
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace

int launch_refine(const FieldDev* fds, const double* const* times, const double* t_ref,
                  const double* grid, int storage, bool optimise, const float* theta,
                  const int32_t* centre, const int32_t* field, const st_candidate* cand,
                  int64_t n, int steps, float fwhm, float lr_pos, float lr_vel, float* J,
                  float* snr, float* grad, st_refined* out, cudaStream_t s) {
  if (n <= 0) return 0;
  RefineArgs a{};
  a.fds = fds;
  a.times = times;
  a.t_ref = t_ref;
  a.theta_in = theta;
  a.centre_in = centre;
  a.field_in = field;
  a.cand = cand;
  a.grid = grid;
  a.n = n;
  const double sg = fwhm / (2.0 * 1.1774100225154747);  // 2 sqrt(2 ln 2)
  a.inv2s2 = (float)(1.0 / (2.0 * sg * sg));
  a.inv_s2 = (float)(1.0 / (sg * sg));
  a.steps = steps;
  a.lr_pos = lr_pos;
  a.lr_vel = lr_vel;
  a.J = J;
  a.snr = snr;
  a.grad = grad;
  a.out = out;
#define ST_REF(T, O) k_refine<T, O><<<(unsigned)n, kThreads, 0, s>>>(a)
  if (storage == ST_F32) {
    if (optimise) ST_REF(float, true); else ST_REF(float, false);
  } else if (storage == ST_F16) {
    if (optimise) ST_REF(__half, true); else ST_REF(__half, false);
  } else {
    if (optimise) ST_REF(__nv_bfloat16, true); else ST_REF(__nv_bfloat16, false);
  }
#undef ST_REF
  return 1;
}

}  // namespace st
