// k_median_select.cu — median star removal (Sec. 2.1) for groups of at most
// 64 frames, one kernel per group size.
//
// The per-pixel median over the group's finite samples (NaN marks a masked
// pixel; an even count takes (a + b) * 0.5 of the two middle values; no
// finite sample gives NaN) is subtracted from every frame of the group.
//
// A block of 128 threads takes 128 consecutive pixels: their columns of N
// frames are copied into shared memory with per-thread asynchronous copies
// (each warp request covers 32 consecutive pixels of one frame), so the cube
// is read from global memory once and the subtraction takes its inputs from
// shared memory.  Each thread turns its column into integer keys that order
// like the floats and sorts them with a bitonic network whose every index is
// a compile-time constant; with N a template constant, the padding of the
// network to a power of two is made of constant keys, so the comparators
// that only move them vanish at compile time, and only those that feed the
// three middle outputs k1 - 1, k1, k1 + 1 (k1 = (N - 1) / 2) remain.
// Masked samples do not change those positions: of a pixel's N - n masked
// samples, half (rounded down) become the lowest key and the rest the
// highest, so the n finite values sit in the middle of the sorted column and
// their one or two middle values fall on k1 - 1 .. k1 + 1:
//   n, N of equal parity: k1 (N odd) or k1, k1 + 1 (N even);
//   n even, N odd: k1 - 1, k1;   n odd, N even: k1.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <array>
#include <utility>

#include "st_internal.h"

namespace st {

namespace {

constexpr int kSelThreads = 128;

// float -> int32 key with the same order (for non-NaN values) and back
__device__ __forceinline__ int32_t to_key(float x) {
  const int32_t b = __float_as_int(x);
  return b ^ ((b >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float from_key(int32_t k) {
  return __int_as_float(k ^ ((k >> 31) & 0x7fffffff));
}

// One stage (k = K, j = J) of the ascending bitonic network over v[0..M),
// then the following stages.
template <int M, int K, int J>
__device__ __forceinline__ void bitonic_keys(int32_t (&v)[M]) {
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int l = i ^ J;
    if (l > i) {
      const int32_t a = v[i], b = v[l];
      const int32_t lo = min(a, b), hi = max(a, b);
      v[i] = (i & K) == 0 ? lo : hi;
      v[l] = (i & K) == 0 ? hi : lo;
    }
  }
  if constexpr (J > 1) {
    bitonic_keys<M, K, J / 2>(v);
  } else if constexpr (K < M) {
    bitonic_keys<M, 2 * K, K>(v);
  }
}

constexpr int pow2_at_least(int n) {
  int m = 1;
  while (m < n) m *= 2;
  return m;
}

template <int N>
__global__ void __launch_bounds__(kSelThreads, 4)
    k_median_select(const float* in, int64_t P, float* out, float* __restrict__ median) {
  constexpr int M = pow2_at_least(N < 2 ? 2 : N);
  __shared__ float col[N][kSelThreads];
  const int tid = threadIdx.x;
  const int64_t p = (int64_t)blockIdx.x * kSelThreads + tid;
  const bool ok = p < P;
  // the columns of the block's pixels (a pixel past the end reads zeros)
  const uint32_t dst0 = (uint32_t)__cvta_generic_to_shared(&col[0][tid]);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float* src = ok ? in + (int64_t)i * P + p : in;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                     dst0 + (uint32_t)(i * kSelThreads * 4)),
                 "l"(src), "r"(ok ? 4 : 0)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  // a thread reads back only what it copied itself; masked samples take
  // the highest and lowest keys alternately (the first the highest)
  int32_t key[M];
  int masked = 0;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    if (i < N) {
      const float x = col[i][tid];
      const bool fin = isfinite(x);
      key[i] = fin ? to_key(x) : ((masked & 1) ? INT32_MIN : INT32_MAX);
      masked += !fin;
    } else {
      key[i] = INT32_MAX;
    }
  }
  bitonic_keys<M, 2, 1>(key);
  constexpr int k1 = (N - 1) / 2;
  const int n = N - masked;
  float med = __int_as_float(0x7fc00000);  // NaN: no finite sample
  if (n > 0) {
    const float lo = from_key(key[k1 > 0 ? k1 - 1 : 0]), mid = from_key(key[k1]);
    const float hi = from_key(key[k1 + 1 < M ? k1 + 1 : k1]);
    if ((n & 1) && (((N ^ n) & 1) == 0 || (N & 1) == 0)) {
      med = mid;                                            // one middle value at k1
    } else if ((N & 1) == 0) {
      med = __fmul_rn(__fadd_rn(mid, hi), 0.5f);            // N, n even
    } else {
      med = __fmul_rn(__fadd_rn(lo, mid), 0.5f);            // N odd, n even
    }
  }
  if (!ok) return;
  if (median) median[p] = med;
#pragma unroll
  for (int i = 0; i < N; ++i) out[(int64_t)i * P + p] = __fsub_rn(col[i][tid], med);
}

using SelectFn = void (*)(const float*, int64_t, float*, float*);

template <int... I>
constexpr auto select_table(std::integer_sequence<int, I...>) {
  return std::array<SelectFn, sizeof...(I)>{{k_median_select<I + 1>...}};
}

}  // namespace

int median_select_max_frames() { return 64; }

int launch_median_select(const float* in, int N, int64_t P, float* out, float* median,
                         cudaStream_t s) {
  static const auto table = select_table(std::make_integer_sequence<int, 64>{});
  if (N < 1 || N > 64) return -1;
  const int64_t blocks = (P + kSelThreads - 1) / kSelThreads;
  if (blocks > 0x7fffffff) return -1;
  table[N - 1]<<<(unsigned)blocks, kSelThreads, 0, s>>>(in, P, out, median);
  return 1;
}

}  // namespace st
