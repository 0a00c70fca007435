// k_stack_generic.cu — direct-gather shift-and-stack kernels (nearest and
// bilinear) for any grid: every sample is read from the L1/L2-cached cube.
// Used where the register-window kernel does not fit the field's motion
// spans, for bilinear mode, and as the plain form the fast kernel is
// measured against.
//
// S_k(x, y) = sum over i = 0..N-1, in order, of I_i(x + sx(i,a), y + sy(i,b))
// (Sec. 1 / Sec. 2.1: each frame shifted along the trial linear motion and
// summed), one FP32 accumulator per output, out-of-frame samples add 0.
#include "st_internal.h"
#include "st_pending.cuh"
#include "st_sample.cuh"

namespace st {

namespace {

constexpr int kTX = 32, kTY = 8, kVG = 8;

template <typename T, int MODE>
__global__ void __launch_bounds__(kTX* kTY)
    k_stack_generic(FieldDev fd, int k0, int nk, const int32_t* __restrict__ dump_k,
                    float* __restrict__ dump_S, int32_t* __restrict__ dump_C,
                    Pending* __restrict__ pend, int64_t cap, Counters* __restrict__ ctr,
                    int tile0) {
  const int W = fd.W, H = fd.H, N = fd.N;
  const int tiles_x = (W + kTX - 1) / kTX;
  const int tile = tile0 + (int)blockIdx.y;
  const int x = (tile % tiles_x) * kTX + (threadIdx.x & 31);
  const int y = (tile / tiles_x) * kTY + (threadIdx.x >> 5);
  const bool pix_ok = x < W && y < H;
  const T* cube = (const T*)fd.cube;
  const int64_t P = (int64_t)W * H;

  int ka[kVG], kb[kVG], kidx[kVG];
  bool kok[kVG];
#pragma unroll
  for (int v = 0; v < kVG; ++v) {
    int q = blockIdx.x * kVG + v;
    kok[v] = q < nk;
    int k = kok[v] ? (dump_k ? dump_k[q] : k0 + q) : 0;
    kidx[v] = k;
    ka[v] = k % fd.nvx;
    kb[v] = k / fd.nvx;
  }
  float acc[kVG];
  int cov[kVG];
#pragma unroll
  for (int v = 0; v < kVG; ++v) { acc[v] = 0.0f; cov[v] = 0; }

  for (int i = 0; i < N; ++i) {
    const T* fr = cube + (int64_t)i * P;
#pragma unroll
    for (int v = 0; v < kVG; ++v) {
      int sx = __ldg(fd.sx + (int64_t)i * fd.nvx + ka[v]);
      int sy = __ldg(fd.sy + (int64_t)i * fd.nvy + kb[v]);
      int u = x + sx, w = y + sy;
      if (MODE == ST_NEAREST) {
        bool in = u >= 0 && w >= 0 && u < W && w < H;
        float s = in ? load_px<T>(fr + (int64_t)w * W + u) : 0.0f;
        acc[v] = __fadd_rn(acc[v], s);
        cov[v] += in;
      } else {
        float fx = __ldg(fd.fx + (int64_t)i * fd.nvx + ka[v]);
        float fy = __ldg(fd.fy + (int64_t)i * fd.nvy + kb[v]);
        BW wt = bilinear_weights(fx, fy);
        acc[v] = bilinear_acc(acc[v], wt, tap<T>(fr, W, H, u, w), tap<T>(fr, W, H, u + 1, w),
                              tap<T>(fr, W, H, u, w + 1), tap<T>(fr, W, H, u + 1, w + 1));
        cov[v] += bilinear_inside(u, fx, W) && bilinear_inside(w, fy, H);
      }
    }
  }

#pragma unroll
  for (int v = 0; v < kVG; ++v) {
    bool ok = pix_ok && kok[v];
    if (dump_S) {
      if (ok) {
        int64_t o = (int64_t)(blockIdx.x * kVG + v) * P + (int64_t)y * W + x;
        dump_S[o] = acc[v];
        if (dump_C) dump_C[o] = cov[v];
      }
      continue;
    }
    bool pass = ok && cov[v] >= fd.nmin && acc[v] >= __ldg(fd.thr + cov[v]);
    Pending rec{x, y, kidx[v], fd.field, acc[v], cov[v]};
    push_pending(pass, rec, pend, cap, ctr);
  }
}

}  // namespace

int launch_stack_generic(const FieldDev& fd, int mode, int k0, int nk, const int32_t* dump_k,
                         float* dump_S, int32_t* dump_C, Pending* pend, int64_t pend_cap,
                         Counters* ctr, cudaStream_t s) {
  if (nk <= 0) return 0;
  int tiles = ((fd.W + kTX - 1) / kTX) * ((fd.H + kTY - 1) / kTY);
  dim3 block(kTX * kTY);
  int launches = 0;
  for (int t0 = 0; t0 < tiles; t0 += 65535) {
    dim3 grid((nk + kVG - 1) / kVG, tiles - t0 < 65535 ? tiles - t0 : 65535);
#define ST_GEN(T, M)                                                                          \
  k_stack_generic<T, M><<<grid, block, 0, s>>>(fd, k0, nk, dump_k, dump_S, dump_C, pend,      \
                                               pend_cap, ctr, t0)
    if (mode == ST_NEAREST) {
      if (fd.storage == ST_F32) ST_GEN(float, ST_NEAREST);
      else if (fd.storage == ST_F16) ST_GEN(__half, ST_NEAREST);
      else ST_GEN(__nv_bfloat16, ST_NEAREST);
    } else {
      if (fd.storage == ST_F32) ST_GEN(float, ST_BILINEAR);
      else if (fd.storage == ST_F16) ST_GEN(__half, ST_BILINEAR);
      else ST_GEN(__nv_bfloat16, ST_BILINEAR);
    }
#undef ST_GEN
    ++launches;
  }
  return launches;
}

}  // namespace st
