// k_prep.cu — time offsets and shift tables (FP64), robust per-frame sky
// statistics (FP64, deterministic) and normalisation into the storage cube.
//
// Shift tables: linear motion with no position-angle constraint (Sec. 2.1):
// frame i is sampled at p + v*dt_i, dt_i = t_i - t_ref, v = v0 + a*dv.  Every
// FP64 operation is an explicit _rn intrinsic so no multiply-add is fused.
//
// Sky statistics: the per-frame sky level and standard deviation used for
// frame QC in Sec. 2.1, read as a kappa-sigma clipped mean and population
// standard deviation (kappa = 3, at most 5 statistics, stop when the kept set
// is unchanged).  Reductions use fixed-order block partials so results do not
// depend on scheduling.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "st_internal.h"

namespace st {

namespace {

__global__ void k_shift_tables(const double* __restrict__ t, int N, double t_ref, double v0,
                               double dv, int nv, int mode, int32_t* __restrict__ s,
                               float* __restrict__ f) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)N * nv) return;
  int i = (int)(idx / nv), a = (int)(idx % nv);
  double dt = __dsub_rn(t[i], t_ref);
  double v = __dadd_rn(v0, __dmul_rn((double)a, dv));
  double p = __dmul_rn(v, dt);
  if (mode == ST_NEAREST) {
    s[idx] = (int32_t)floor(__dadd_rn(p, 0.5));
    if (f) f[idx] = 0.0f;
  } else {
    double fl = floor(p);
    s[idx] = (int32_t)fl;
    if (f) f[idx] = (float)__dsub_rn(p, fl);
  }
}

constexpr int kSkyBlocks = 64;    // partial sums per frame
constexpr int kSkyThreads = 256;
constexpr int kSkyIters = 5;
constexpr double kKappa = 3.0;

// Per-frame state: [0] mu, [1] sigma, [2] mu_prev, [3] sigma_prev, [4] done,
// [5] iteration count, [6] kept count.
constexpr int kState = 8;

struct Acc4 {
  double n, s1, s2, ch;
};

__device__ inline Acc4 block_reduce4(Acc4 v, double* sh) {
  // fixed-order tree over the block (deterministic)
  int tid = threadIdx.x;
  sh[tid * 4 + 0] = v.n;
  sh[tid * 4 + 1] = v.s1;
  sh[tid * 4 + 2] = v.s2;
  sh[tid * 4 + 3] = v.ch;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w)
      for (int q = 0; q < 4; ++q) sh[tid * 4 + q] = __dadd_rn(sh[tid * 4 + q], sh[(tid + w) * 4 + q]);
    __syncthreads();
  }
  Acc4 r{sh[0], sh[1], sh[2], sh[3]};
  return r;
}

// pass kind 0: count and sum of finite pixels.
// pass kind 1: sum of (x - mu)^2 over finite pixels (mu from state).
// pass kind 2: clipped pass: membership with (mu, sigma) of the previous
//   statistics, pivot p = mu; accumulates n, sum(x-p), sum((x-p)^2) and the
//   number of pixels whose membership changed against the set before.
__global__ void k_sky_pass(const float* __restrict__ raw, int64_t npix, int kind,
                           int first_clip, const double* __restrict__ state,
                           double* __restrict__ partial) {
  __shared__ double sh[kSkyThreads * 4];
  int i = blockIdx.y;
  const double* st = state + (int64_t)i * kState;
  if (st[4] != 0.0) return;  // frame converged (uniform per block)
  const float* x = raw + (int64_t)i * npix;
  double mu = st[0], sg = st[1], mup = st[2], sgp = st[3];
  double thr = __dmul_rn(kKappa, sg), thrp = __dmul_rn(kKappa, sgp);
  Acc4 a{0, 0, 0, 0};
  int64_t chunk = (npix + gridDim.x - 1) / gridDim.x;
  int64_t j0 = (int64_t)blockIdx.x * chunk;
  int64_t j1 = min(npix, j0 + chunk);
  for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    float xf = x[j];
    if (!isfinite(xf)) continue;
    double xv = (double)xf;
    if (kind == 0) {
      a.n += 1.0;
      a.s1 = __dadd_rn(a.s1, xv);
    } else if (kind == 1) {
      double d = __dsub_rn(xv, mu);
      a.s2 = __dadd_rn(a.s2, __dmul_rn(d, d));
    } else {
      double d = __dsub_rn(xv, mu);
      bool keep = fabs(d) <= thr;
      bool keep_before = first_clip ? true : (fabs(__dsub_rn(xv, mup)) <= thrp);
      if (keep != keep_before) a.ch += 1.0;
      if (keep) {
        a.n += 1.0;
        a.s1 = __dadd_rn(a.s1, d);
        a.s2 = __dadd_rn(a.s2, __dmul_rn(d, d));
      }
    }
  }
  Acc4 r = block_reduce4(a, sh);
  if (threadIdx.x == 0) {
    double* p = partial + ((int64_t)i * kSkyBlocks + blockIdx.x) * 4;
    p[0] = r.n;
    p[1] = r.s1;
    p[2] = r.s2;
    p[3] = r.ch;
  }
}

// One block per frame: reduce the partials in fixed order and update the state.
__global__ void k_sky_finalize(int kind, int iter, double* __restrict__ state,
                               const double* __restrict__ partial) {
  __shared__ double sh[kSkyBlocks * 4];
  int i = blockIdx.x;
  double* st = state + (int64_t)i * kState;
  if (st[4] != 0.0) return;
  Acc4 v{0, 0, 0, 0};
  if (threadIdx.x < kSkyBlocks) {
    const double* p = partial + ((int64_t)i * kSkyBlocks + threadIdx.x) * 4;
    v = Acc4{p[0], p[1], p[2], p[3]};
  }
  Acc4 r = block_reduce4(v, sh);
  if (threadIdx.x != 0) return;
  if (kind == 0) {
    st[6] = r.n;
    st[0] = r.n > 0 ? __ddiv_rn(r.s1, r.n) : 0.0;
    if (r.n == 0) { st[1] = 0.0; st[4] = 1.0; st[5] = 1.0; }
  } else if (kind == 1) {
    st[1] = st[6] > 0 ? __dsqrt_rn(__ddiv_rn(r.s2, st[6])) : 0.0;
    st[5] = 1.0;
    if (iter >= kSkyIters) st[4] = 1.0;
  } else {
    if (r.ch == 0.0 || r.n == 0.0) {  // kept set unchanged: keep the last statistics
      st[4] = 1.0;
      return;
    }
    double p = st[0];
    double m1 = __ddiv_rn(r.s1, r.n);
    double mu = __dadd_rn(p, m1);
    double var = __dsub_rn(__ddiv_rn(r.s2, r.n), __dmul_rn(m1, m1));
    st[2] = st[0];
    st[3] = st[1];
    st[0] = mu;
    st[1] = __dsqrt_rn(var > 0.0 ? var : 0.0);
    st[5] = (double)iter;
    st[6] = r.n;
    if (iter >= kSkyIters) st[4] = 1.0;
  }
}

template <typename T>
__device__ inline T to_store(float v);
template <>
__device__ inline float to_store<float>(float v) { return v; }
template <>
__device__ inline __half to_store<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ inline __nv_bfloat16 to_store<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// I = (R - mu) * (1/sigma) in FP64, rounded to FP32; NaN -> 0; optional clip.
template <typename T>
__global__ void k_normalize_store(const float* __restrict__ raw, int64_t npix, int normalize,
                                  float cr_clip, const double* __restrict__ state,
                                  T* __restrict__ cube, double* __restrict__ mu_out,
                                  double* __restrict__ sigma_out) {
  int i = blockIdx.y;
  const float* x = raw + (int64_t)i * npix;
  T* o = cube + (int64_t)i * npix;
  double mu = 0.0, inv = 1.0;
  bool zero = false;
  if (normalize) {
    const double* st = state + (int64_t)i * kState;
    mu = st[0];
    double sg = st[1];
    zero = !(sg > 0.0);
    inv = zero ? 0.0 : __drcp_rn(sg);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (mu_out) mu_out[i] = mu;
      if (sigma_out) sigma_out[i] = sg;
    }
  }
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < npix; j += stride) {
    float r = x[j];
    float v;
    if (normalize) {
      v = 0.0f;
      if (isfinite(r) && !zero) v = (float)__dmul_rn(__dsub_rn((double)r, mu), inv);
      if (cr_clip > 0.0f && fabsf(v) > cr_clip) v = 0.0f;
    } else {
      v = r;
    }
    o[j] = to_store<T>(v);
  }
}

__global__ void k_sky_init(double* state, int N) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int q = 0; q < kState; ++q) state[(int64_t)i * kState + q] = 0.0;
}

}  // namespace

int launch_shift_tables(const double* d_t, int N, double t_ref, double vx0, double dvx, int nvx,
                        double vy0, double dvy, int nvy, int mode, int32_t* sx, int32_t* sy,
                        float* fx, float* fy, cudaStream_t s) {
  int64_t nx = (int64_t)N * nvx, ny = (int64_t)N * nvy;
  k_shift_tables<<<(unsigned)((nx + 255) / 256), 256, 0, s>>>(d_t, N, t_ref, vx0, dvx, nvx, mode,
                                                               sx, fx);
  k_shift_tables<<<(unsigned)((ny + 255) / 256), 256, 0, s>>>(d_t, N, t_ref, vy0, dvy, nvy, mode,
                                                               sy, fy);
  return 2;
}

size_t sky_partial_doubles(int N) {
  return (size_t)N * kSkyBlocks * 4 + (size_t)N * kState;
}

int launch_normalize(const float* raw, int N, int64_t npix, int normalize, float cr_clip,
                     int storage, void* cube, double* mu, double* sigma, double* partial,
                     cudaStream_t s) {
  int launches = 0;
  double* state = partial + (size_t)N * kSkyBlocks * 4;
  if (normalize) {
    k_sky_init<<<(N + 127) / 128, 128, 0, s>>>(state, N);
    dim3 g(kSkyBlocks, N);
    k_sky_pass<<<g, kSkyThreads, 0, s>>>(raw, npix, 0, 0, state, partial);
    k_sky_finalize<<<N, kSkyBlocks, 0, s>>>(0, 1, state, partial);
    k_sky_pass<<<g, kSkyThreads, 0, s>>>(raw, npix, 1, 0, state, partial);
    k_sky_finalize<<<N, kSkyBlocks, 0, s>>>(1, 1, state, partial);
    launches += 5;
    for (int it = 2; it <= kSkyIters; ++it) {
      k_sky_pass<<<g, kSkyThreads, 0, s>>>(raw, npix, 2, it == 2 ? 1 : 0, state, partial);
      k_sky_finalize<<<N, kSkyBlocks, 0, s>>>(2, it, state, partial);
      launches += 2;
    }
  }
  int bx = (int)((npix + 256 * 8 - 1) / (256 * 8));
  if (bx > 1024) bx = 1024;
  if (bx < 1) bx = 1;
  dim3 g(bx, N);
  switch (storage) {
    case ST_F32:
      k_normalize_store<float><<<g, 256, 0, s>>>(raw, npix, normalize, cr_clip, state,
                                                 (float*)cube, mu, sigma);
      break;
    case ST_F16:
      k_normalize_store<__half><<<g, 256, 0, s>>>(raw, npix, normalize, cr_clip, state,
                                                  (__half*)cube, mu, sigma);
      break;
    default:
      k_normalize_store<__nv_bfloat16><<<g, 256, 0, s>>>(raw, npix, normalize, cr_clip, state,
                                                         (__nv_bfloat16*)cube, mu, sigma);
      break;
  }
  return launches + 1;
}

}  // namespace st
