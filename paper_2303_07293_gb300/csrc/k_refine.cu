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
// every evaluation, never stored.  A frame's shift v dt_i is formed to
// FP64 accuracy (the time offset held as an FP32 pair, the product with an
// exact FMA error term) and split into its integer part and FP32 fraction.
//
// Optimisers (maximise J with F at its optimum <g,S>/(N <g,g>) each step):
// Adam on (vx, vy, x0, y0), or Gauss-Newton: J is the log-likelihood of the
// frames under the model F g(p - (x0, y0) - v dt_i), so -Hessian is replaced
// by the model's J^T J, whose entries need only template sums over the
// cutout (<g,g>, <g,Gx>, <g,Gy>, <Gx,Gx>, <Gy,Gy>, <Gx,Gy> with G = dg/dx0,
// dg/dy0) and sum dt, sum dt^2; F is profiled out by the Schur complement of
// its entry and (vx, vy, x0, y0) move by the solution of
// (Hs + damping diag(Hs)) delta = dJ/d(vx, vy, x0, y0).
//
// One CTA per candidate.  Every pixel of the cutout shares a frame's shift,
// so a frame contributes one footprint of 65 x 65 taps; a TMA ring of S
// frames stages those footprints in shared memory ahead of use (zero fill
// outside the image takes the place of bounds tests; the box x origin is
// rounded down to 16 bytes and the remainder is an index offset).  Thread t
// owns cutout column t%64 and its 16 rows (t/64)*16.., so a warp reads 32
// consecutive words of a box row; it walks its rows with the horizontal
// interpolation h = a0 + fx (a1 - a0) of the row below carried over, so each
// tap row is read and interpolated once.  Reductions use a fixed-order block
// tree.  Every wait is bounded in time.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <vector>

#include "st_internal.h"
#include "st_sample.cuh"
#include "st_tma.cuh"

namespace st {

namespace {

constexpr int kCut = 64;        // cutout side
constexpr int kThreads = 256;
constexpr int kPix = kCut * kCut / kThreads;  // 16 rows of one column per thread
constexpr int kSums = 11;
constexpr int kBoxW = 72;       // footprint columns: 65 taps + up to 7 of alignment
constexpr int kBoxH = kCut + 1; // footprint rows
constexpr uint64_t kWaitNs = 2000000000ull;  // wait limit: 2 s of wall-clock time

template <typename T>
constexpr int stages_for() { return sizeof(T) == 4 ? 4 : 6; }
template <typename T>
constexpr int box_bytes() { return ((kBoxW * kBoxH * (int)sizeof(T)) + 127) & ~127; }
template <typename T>
constexpr int align_elems() { return 16 / (int)sizeof(T); }

struct RefineArgs {
  const FieldDev* fds;          // device field descriptors
  const CUtensorMap* maps;      // per field: tiled map of the cube, box kBoxW x kBoxH x 1
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
  int optimizer;                // 0: Adam, 1: Gauss-Newton (optimise mode)
  float lr_pos, lr_vel;         // Adam learning rates; Gauss-Newton: lr_pos = damping
  float* J;
  float* snr;
  float* grad;                  // [n][5] or null
  st_refined* out;              // optimise mode
  int* err;                     // timeout flag
};

template <typename T>
__device__ __forceinline__ float ld_s(const T* p);
template <>
__device__ __forceinline__ float ld_s<float>(const float* p) { return *p; }
template <>
__device__ __forceinline__ float ld_s<__half>(const __half* p) { return __half2float(*p); }
template <>
__device__ __forceinline__ float ld_s<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
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

// A frame's shift for velocity (vx, vy): integer parts and fractions.
struct Shift {
  int ux, uy;
  float fx, fy;
};
// floor and fraction of v (dt_hi + dt_lo) without FP64 arithmetic: p = fl(v
// dt_hi) and its exact rounding error (one FMA) plus v dt_lo give the product
// as p + q to about 2^-46 relative; p - floor(p) is exact below 2^23 px, and
// the fraction is (p - floor(p)) + q rounded to FP32, moved into [0, 1).
__device__ __forceinline__ void split_shift(float v, float dt_hi, float dt_lo, int* u, float* f) {
  const float p = v * dt_hi;
  const float q = __fmaf_rn(v, dt_lo, __fmaf_rn(v, dt_hi, -p));
  float fl = floorf(p);
  float r = (p - fl) + q;
  if (r < 0.0f) {
    fl -= 1.0f;
    r += 1.0f;
  } else if (r >= 1.0f) {
    fl += 1.0f;
    r -= 1.0f;
  }
  *u = (int)fl;
  *f = r;
}
__device__ __forceinline__ Shift frame_shift(float vx, float vy, float dt_hi, float dt_lo) {
  Shift s;
  split_shift(vx, dt_hi, dt_lo, &s.ux, &s.fx);
  split_shift(vy, dt_hi, dt_lo, &s.uy, &s.fy);
  return s;
}

// Solves the 4 x 4 system A x = b by Gaussian elimination with partial
// pivoting (FP64, in place).  Returns false for a (near) singular matrix.
__device__ bool solve4(double (&A)[4][4], double (&b)[4]) {
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (!(fabs(A[piv][c]) > 1e-300)) return false;
    if (piv != c) {
      for (int k = 0; k < 4; ++k) {
        const double tmp = A[c][k];
        A[c][k] = A[piv][k];
        A[piv][k] = tmp;
      }
      const double tb = b[c];
      b[c] = b[piv];
      b[piv] = tb;
    }
    for (int r = c + 1; r < 4; ++r) {
      const double f = A[r][c] / A[c][c];
      for (int k = c; k < 4; ++k) A[r][k] -= f * A[c][k];
      b[r] -= f * b[c];
    }
  }
  for (int c = 3; c >= 0; --c) {
    double v = b[c];
    for (int k = c + 1; k < 4; ++k) v -= A[c][k] * b[k];
    b[c] = v / A[c][c];
  }
  return true;
}

// One Gauss-Newton step of (vx, vy, x0, y0) (in th[0..3]) at flux F from the
// block sums s (template sums s[1] = <g,g>, s[4] = <g,Gx>, s[5] = <g,Gy>,
// s[8] = <Gx,Gx>, s[9] = <Gy,Gy>, s[10] = <Gx,Gy>), the gradient gr and the
// frames' sum dt and sum dt^2.  A singular system leaves th unchanged.
__device__ void gauss_newton_step(float* th, const float (&s)[kSums], const float (&gr)[5],
                                  float F, int N, double T1, double T2, float damping) {
  const double f = F, f2 = f * f, n = N;
  const double xx = s[8], yy = s[9], xy = s[10], gx = s[4], gy = s[5], gg = s[1];
  const double H[5][5] = {{f2 * T2 * xx, f2 * T2 * xy, f2 * T1 * xx, f2 * T1 * xy, f * T1 * gx},
                          {f2 * T2 * xy, f2 * T2 * yy, f2 * T1 * xy, f2 * T1 * yy, f * T1 * gy},
                          {f2 * T1 * xx, f2 * T1 * xy, f2 * n * xx, f2 * n * xy, f * n * gx},
                          {f2 * T1 * xy, f2 * T1 * yy, f2 * n * xy, f2 * n * yy, f * n * gy},
                          {f * T1 * gx, f * T1 * gy, f * n * gx, f * n * gy, n * gg}};
  if (!(H[4][4] > 0.0)) return;
  double A[4][4], b[4];
  for (int a = 0; a < 4; ++a) {
    for (int c = 0; c < 4; ++c) A[a][c] = H[a][c] - H[a][4] * H[4][c] / H[4][4];
    b[a] = gr[a];
  }
  for (int a = 0; a < 4; ++a) A[a][a] += (double)damping * A[a][a];
  if (!solve4(A, b)) return;
  for (int a = 0; a < 4; ++a) th[a] = (float)((double)th[a] + b[a]);
}

template <typename T, bool OPT>
__global__ void __launch_bounds__(kThreads, 2) k_refine(RefineArgs a) {
  constexpr int S = stages_for<T>();
  constexpr int kBox = box_bytes<T>();
  constexpr int kAl = align_elems<T>();
  extern __shared__ __align__(128) unsigned char dsm_raw[];
  __shared__ __align__(8) uint64_t full[S];
  __shared__ float sh[(kThreads / 32) * kSums];
  __shared__ float th[5];
  __shared__ double s_t12[2];   // sum dt, sum dt^2 (Gauss-Newton)
  __shared__ int s_ok;
  unsigned char* ring = dsm_raw + ((128u - (smem_u32(dsm_raw) & 127u)) & 127u);
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
  const int N = fd.N;
  // time offsets dt_i = t_i - t_ref as FP32 pairs: sdt (rounded) + sdt_lo
  float* sdt = reinterpret_cast<float*>(ring + (size_t)S * kBox);
  float* sdt_lo = sdt + N;
  const CUtensorMap* map = a.maps + fi;
  const int tid = threadIdx.x;
  const bool gn = OPT && a.optimizer == 1;
  {
    const double* t = a.times[fi];
    const double t_ref = a.t_ref[fi];
    double p1 = 0.0, p2 = 0.0;
    for (int j = tid; j < N; j += kThreads) {
      const double d = t[j] - t_ref;
      sdt[j] = (float)d;
      sdt_lo[j] = (float)(d - (double)(float)d);
      p1 += d;
      p2 += d * d;
    }
    if (gn) {
      // sum dt and sum dt^2 in FP64, fixed-order block reduction
      for (int d = 16; d > 0; d >>= 1) {
        p1 += __shfl_down_sync(0xffffffffu, p1, d);
        p2 += __shfl_down_sync(0xffffffffu, p2, d);
      }
      __shared__ double s_p[2 * (kThreads / 32)];
      if ((tid & 31) == 0) {
        s_p[2 * (tid >> 5)] = p1;
        s_p[2 * (tid >> 5) + 1] = p2;
      }
      __syncthreads();
      if (tid == 0) {
        double a1 = 0.0, a2 = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
          a1 += s_p[2 * w];
          a2 += s_p[2 * w + 1];
        }
        s_t12[0] = a1;
        s_t12[1] = a2;
      }
    }
  }
  if (tid == 0) {
    tma_prefetch_desc(map);
    for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
    mbar_init_fence();
    s_ok = 1;
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

  // thread 0 stages frame i (sequence number q) into ring slot q % S
  uint32_t q_issued = 0;  // (thread 0) sequence number after the last staged frame
  auto issue = [&](int i, uint32_t q, float vx, float vy) {
    q_issued = q + 1;
    const Shift f = frame_shift(vx, vy, sdt[i], sdt_lo[i]);
    const int cu0 = cx - kCut / 2 + f.ux, cv0 = cy - kCut / 2 + f.uy;
    const int bx = cu0 & ~(kAl - 1);  // 16-byte aligned box origin (floor, also below 0)
    const int slot = (int)(q % S);
    mbar_arrive_expect_tx(&full[slot], (uint32_t)(kBoxW * kBoxH * sizeof(T)));
    tma_load_3d(ring + (size_t)slot * kBox, map, bx, cv0, i, &full[slot]);
  };

  const int col = tid % kCut;
  const int row0 = (tid / kCut) * kPix;
  const float fcol = (float)(cx - kCut / 2 + col);
  const float frow0 = (float)(cy - kCut / 2 + row0);
  float sums[kSums];
  float m[4] = {0, 0, 0, 0}, v2[4] = {0, 0, 0, 0};
  const int steps = OPT ? a.steps : 0;
  uint32_t q0 = 0;  // frames staged before this evaluation
  bool ok = true;
  for (int step = 0; step <= steps && ok; ++step) {
    const float vx = th[0], vy = th[1], x0 = th[2], y0 = th[3];
    if (tid == 0)
      for (int i = 0; i < S && i < N; ++i) issue(i, q0 + i, vx, vy);
    float S_[kPix], g[kPix];
    const float dx = fcol - x0;
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
      S_[k] = 0.0f;
      const float dy = frow0 + (float)k - y0;
      g[k] = expf(-(dx * dx + dy * dy) * a.inv2s2);
    }
    float dvx = 0.0f, dvy = 0.0f;
    for (int i = 0; i < N; ++i) {
      const uint32_t q = q0 + i;
      const int slot = (int)(q % S);
      if (!mbar_wait(&full[slot], (q / S) & 1u, kWaitNs)) {
        atomicOr(a.err, 1);
        s_ok = 0;
      }
      const float dt = sdt[i];
      const Shift f = frame_shift(vx, vy, dt, sdt_lo[i]);
      const int cu0 = cx - kCut / 2 + f.ux;
      const T* box = reinterpret_cast<const T*>(ring + (size_t)slot * kBox) +
                     (size_t)row0 * kBoxW + (cu0 - (cu0 & ~(kAl - 1))) + col;
      float a0 = ld_s<T>(box), a1 = ld_s<T>(box + 1);
      float dp = a1 - a0;        // a1 - a0 of the row above
      float hp = a0 + f.fx * dp; // its horizontal interpolation (top)
      float gdx = 0.0f, gdy = 0.0f;
#pragma unroll
      for (int k = 0; k < kPix; ++k) {
        const T* r = box + (k + 1) * kBoxW;
        const float b0 = ld_s<T>(r), b1 = ld_s<T>(r + 1);
        const float d = b1 - b0;
        const float h = b0 + f.fx * d;   // bottom
        const float dh = h - hp;         // bot - top
        S_[k] += hp + f.fy * dh;
        gdx += g[k] * (dp + f.fy * (d - dp));  // (1-fy)(a1-a0) + fy(b1-b0)
        gdy += g[k] * dh;
        hp = h;
        dp = d;
      }
      dvx += dt * gdx;
      dvy += dt * gdy;
      __syncthreads();  // every thread is done with the slot
      if (!s_ok) {
        ok = false;
        break;
      }
      if (tid == 0 && i + S < N) issue(i + S, q + S, vx, vy);
    }
    if (!ok) break;
    q0 += (uint32_t)N;
#pragma unroll
    for (int k = 0; k < kSums; ++k) sums[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
      const float dy = frow0 + (float)k - y0;
      const float gx = g[k] * dx * a.inv_s2;
      const float gy = g[k] * dy * a.inv_s2;
      sums[0] += g[k] * S_[k];
      sums[1] += g[k] * g[k];
      sums[2] += gx * S_[k];
      sums[3] += gy * S_[k];
      sums[4] += g[k] * gx;
      sums[5] += g[k] * gy;
      sums[8] += gx * gx;
      sums[9] += gy * gy;
      sums[10] += gx * gy;
    }
    sums[6] = dvx;
    sums[7] = dvy;
    block_sum(sums, sh);
    if (tid == 0) {
      // F at its optimum <g,S>/(N <g,g>) when optimising (profile likelihood)
      if (OPT) th[4] = sums[1] > 0.0f ? sums[0] / ((float)N * sums[1]) : 0.0f;
      float J, snr, gr[5];
      objective(sums, N, th[4], &J, &snr, gr);
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
      } else if (gn) {
        gauss_newton_step(th, sums, gr, th[4], N, s_t12[0], s_t12[1], a.lr_pos);
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
  if (!ok && tid == 0) {
    // a wait gave up: let the copies already issued land (bounded) before
    // exit; only the latest phase of each slot can be waited on
    for (uint32_t q = q_issued > (uint32_t)S ? q_issued - S : 0; q < q_issued; ++q)
      mbar_wait(&full[q % S], (q / S) & 1u, kWaitNs);
  }
}

template <typename T, bool OPT>
void set_smem_attr() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute((const void*)k_refine<T, OPT>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    done = true;
  }
}

}  // namespace

int refine_max_frames() { return 8192; }

int launch_refine(const FieldDev* h_fds, int n_fields, const FieldDev* fds, CUtensorMap* d_maps,
                  const double* const* times, const double* t_ref, const double* grid,
                  int storage, bool optimise, const float* theta, const int32_t* centre,
                  const int32_t* field, const st_candidate* cand, int64_t n, int steps,
                  int optimizer, float fwhm, float lr_pos, float lr_vel, float* J, float* snr,
                  float* grad, st_refined* out, int* err, cudaStream_t s) {
  if (n <= 0) return 0;
  // tensor maps of the fields' cubes (box: the footprint of one frame)
  std::vector<CUtensorMap> maps(n_fields);
  int max_n = 0;
  for (int f = 0; f < n_fields; ++f) {
    if (!encode_tile_map(&maps[f], h_fds[f], kBoxW, kBoxH)) return -1;
    max_n = h_fds[f].N > max_n ? h_fds[f].N : max_n;
  }
  if (max_n > refine_max_frames()) return -1;
  if (cudaMemcpyAsync(d_maps, maps.data(), sizeof(CUtensorMap) * n_fields,
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return -1;
  RefineArgs a{};
  a.fds = fds;
  a.maps = d_maps;
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
  a.optimizer = optimizer;
  a.lr_pos = lr_pos;
  a.lr_vel = lr_vel;
  a.J = J;
  a.snr = snr;
  a.grad = grad;
  a.out = out;
  a.err = err;
  const size_t dt_bytes = 2 * sizeof(float) * (size_t)max_n;
#define ST_REF(T, O)                                                                         \
  do {                                                                                       \
    set_smem_attr<T, O>();                                                                   \
    const size_t smem = (size_t)stages_for<T>() * box_bytes<T>() + dt_bytes + 128;           \
    k_refine<T, O><<<(unsigned)n, kThreads, smem, s>>>(a);                                   \
  } while (0)
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
