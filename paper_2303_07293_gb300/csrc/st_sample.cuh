// st_sample.cuh — per-sample arithmetic shared by every kernel that forms a
// stack value, so the stack kernels and the local-maximum resolver produce
// bit-identical sums (Sec. 1: shift along the motion, then sum the frames).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace st {

template <typename T>
__device__ __forceinline__ float load_px(const T* p);
template <>
__device__ __forceinline__ float load_px<float>(const float* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float load_px<__half>(const __half* p) { return __half2float(__ldg(p)); }
template <>
__device__ __forceinline__ float load_px<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}

// Pixel (u, v) of a frame, 0 outside.
template <typename T>
__device__ __forceinline__ float tap(const T* frame, int W, int H, int u, int v) {
  return (u >= 0 && v >= 0 && u < W && v < H) ? load_px<T>(frame + (int64_t)v * W + u) : 0.0f;
}

// Bilinear weights from the FP32 fractions: (1-fx)(1-fy), fx(1-fy), (1-fx)fy, fx fy,
// each one rounded product.
struct BW {
  float w00, w10, w01, w11;
};
__device__ __forceinline__ BW bilinear_weights(float fx, float fy) {
  float gx = __fsub_rn(1.0f, fx), gy = __fsub_rn(1.0f, fy);
  BW w;
  w.w00 = __fmul_rn(gx, gy);
  w.w10 = __fmul_rn(fx, gy);
  w.w01 = __fmul_rn(gx, fy);
  w.w11 = __fmul_rn(fx, fy);
  return w;
}

// acc + sample, as four fused multiply-adds in the fixed order 00, 10, 01, 11.
__device__ __forceinline__ float bilinear_acc(float acc, const BW& w, float i00, float i10,
                                              float i01, float i11) {
  acc = __fmaf_rn(w.w00, i00, acc);
  acc = __fmaf_rn(w.w10, i10, acc);
  acc = __fmaf_rn(w.w01, i01, acc);
  acc = __fmaf_rn(w.w11, i11, acc);
  return acc;
}

// Bilinear coverage: the sample x + s lies in [0, W-1] with s = floor + fraction.
__device__ __forceinline__ bool bilinear_inside(int u, float f, int W) {
  return u >= 0 && (u <= W - 2 || (u == W - 1 && f == 0.0f));
}

}  // namespace st
