// k_front.cu — the pre-tracking front end of Sec. 2.1 on the device.
//
// * Median star removal: for a group of frames, the per-pixel median over the
//   group (finite values only; NaN marks a masked pixel; an even count takes
//   (a + b) * 0.5 of the two middle values) is subtracted from every frame,
//   removing the stationary high-S/N sources before the shift-and-stack.
// * Frame sums: every n consecutive frames summed in frame order with one
//   FP32 accumulator (a trailing partial group is dropped), for slow movers.
// * 2 x 2 binning: ((p00 + p01) + p10) + p11 per block (flux kept), for fast
//   movers.
//
// All three are HBM-bound streams.  The median kernels give each thread one
// pixel, so a warp reads 32 consecutive pixels of a frame per load
// (coalesced).  Up to 64 frames a sorting network per group size selects the
// median (k_median_select.cu); longer groups keep each pixel's samples in a
// private shared-memory column (lane = bank, no conflicts), copied
// asynchronously, and select the middle values in place by quickselect, the
// untouched copy of the column supplying the subtraction.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "st_internal.h"

namespace st {

namespace {

constexpr int kMedThreads = 32;  // one warp per block; samples in shared memory

// k-th smallest of a[0..n-1] (stride kMedThreads), partially reordering a.
__device__ float quickselect(float* a, int n, int k) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    // median of three as the pivot
    const int mid = lo + (hi - lo) / 2;
    float x = a[lo * kMedThreads], y = a[mid * kMedThreads], z = a[hi * kMedThreads];
    const float piv = fmaxf(fminf(x, y), fminf(fmaxf(x, y), z));
    int i = lo, j = hi;
    while (i <= j) {
      while (a[i * kMedThreads] < piv) ++i;
      while (a[j * kMedThreads] > piv) --j;
      if (i <= j) {
        const float t = a[i * kMedThreads];
        a[i * kMedThreads] = a[j * kMedThreads];
        a[j * kMedThreads] = t;
        ++i;
        --j;
      }
    }
    if (k <= j) hi = j;
    else if (k >= i) lo = i;
    else return a[k * kMedThreads];
  }
  return a[k * kMedThreads];
}

// in and out may be the same cube: a thread copies its pixel's whole column
// before it writes any of it, and no other thread touches that pixel.
__global__ void __launch_bounds__(kMedThreads)
    k_median_subtract(const float* in, int N, int64_t P, float* out,
                      float* __restrict__ median) {
  extern __shared__ float sm[];
  float* orig = sm;                      // [N][32] the pixel's samples in frame order
  float* work = sm + (size_t)N * kMedThreads;  // [n][32] its finite samples, reordered
  const int lane = threadIdx.x;
  const int64_t p = (int64_t)blockIdx.x * kMedThreads + lane;
  const bool ok = p < P;
  // the column, copied asynchronously (all N copies in flight at once; a
  // pixel past the end copies nothing and reads zeros)
  const uint32_t dst0 = (uint32_t)__cvta_generic_to_shared(orig + lane);
  for (int i = 0; i < N; ++i) {
    const float* src = ok ? in + (int64_t)i * P + p : in;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                     dst0 + (uint32_t)(i * kMedThreads * 4)),
                 "l"(src), "r"(ok ? 4 : 0)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  int n = 0;
  for (int i = 0; i < N; ++i) {
    const float v = orig[i * kMedThreads + lane];
    if (isfinite(v)) work[(n++) * kMedThreads + lane] = v;
  }
  float med = __int_as_float(0x7fc00000);  // NaN: no finite sample
  if (n > 0) {
    float* col = work + lane;
    const int k1 = (n - 1) / 2;
    const float a = quickselect(col, n, k1);
    if (n & 1) {
      med = a;
    } else {
      // the next order statistic: the least value above position k1
      float b = col[(k1 + 1) * kMedThreads];
      for (int q = k1 + 2; q < n; ++q) b = fminf(b, col[q * kMedThreads]);
      med = __fmul_rn(__fadd_rn(a, b), 0.5f);
    }
  }
  if (!ok) return;
  if (median) median[p] = med;
  for (int i = 0; i < N; ++i) out[(int64_t)i * P + p] = __fsub_rn(orig[i * kMedThreads + lane], med);
}

__global__ void k_sum_frames(const float* __restrict__ in, int n_sum, int M, int64_t P,
                             float* __restrict__ out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (p >= P || m >= M) return;
  const float* src = in + (int64_t)m * n_sum * P + p;
  float acc = 0.0f;
  for (int i = 0; i < n_sum; ++i) acc = __fadd_rn(acc, src[(int64_t)i * P]);
  out[(int64_t)m * P + p] = acc;
}

__global__ void k_bin2x2(const float* __restrict__ in, int H, int W, int h, int w,
                         float* __restrict__ out) {
  const int X = blockIdx.x * blockDim.x + threadIdx.x;
  const int Y = blockIdx.y;
  const int64_t f = blockIdx.z;
  if (X >= w || Y >= h) return;
  const float* r0 = in + (f * H + 2 * Y) * (int64_t)W + 2 * X;
  const float* r1 = r0 + W;
  out[(f * h + Y) * (int64_t)w + X] =
      __fadd_rn(__fadd_rn(__fadd_rn(r0[0], r0[1]), r1[0]), r1[1]);
}

}  // namespace

int median_max_frames() { return 768; }  // 2 x 768 x 32 floats = 192 KB of shared memory

int launch_median_subtract(const float* in, int N, int64_t P, float* out, float* median,
                           cudaStream_t s) {
  // up to 64 frames: a sorting network per group size (k_median_select.cu)
  if (N <= median_select_max_frames()) return launch_median_select(in, N, P, out, median, s);
  const size_t smem = (size_t)2 * N * kMedThreads * sizeof(float);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute((const void*)k_median_subtract,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * median_max_frames() * kMedThreads * 4);
    attr = true;
  }
  const int64_t blocks = (P + kMedThreads - 1) / kMedThreads;
  if (blocks > 0x7fffffff) return -1;
  k_median_subtract<<<(unsigned)blocks, kMedThreads, smem, s>>>(in, N, P, out, median);
  return 1;
}

int launch_sum_frames(const float* in, int n_sum, int M, int64_t P, float* out, cudaStream_t s) {
  if (M <= 0) return 0;
  const int64_t bx = (P + 255) / 256;
  if (bx > 0x7fffffff || M > 65535) return -1;
  k_sum_frames<<<dim3((unsigned)bx, (unsigned)M), 256, 0, s>>>(in, n_sum, M, P, out);
  return 1;
}

int launch_bin2x2(const float* in, int N, int H, int W, float* out, cudaStream_t s) {
  const int h = H / 2, w = W / 2;
  if (h <= 0 || w <= 0 || N <= 0) return 0;
  if (h > 65535 || N > 65535) return -1;
  k_bin2x2<<<dim3((unsigned)((w + 127) / 128), (unsigned)h, (unsigned)N), 128, 0, s>>>(
      in, H, W, h, w, out);
  return 1;
}

}  // namespace st
