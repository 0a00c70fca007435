// k_probe.cu — FP32 add-rate microbenchmark, the roof of the stack kernels.
//
// One block of 1024 threads per SM runs 16 independent FP32 add chains per
// thread; SM cycles come from clock64 inside each block.  Variants:
//   0: scalar add.rn.f32
//   1: paired add.rn.f32x2 (16 adds as 8 paired instructions)
//   2: paired adds interleaved 1:1 with independent integer adds (tests
//      whether other pipes issue in the paired add's second cycle)
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "st_internal.h"
#include "st_tma.cuh"

namespace st {

namespace {

template <int VAR>
__global__ void __launch_bounds__(1024, 1)
    k_add_rate(const float* __restrict__ in, float* __restrict__ out, int iters,
               long long* __restrict__ cycles) {
  float b[16], a[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    b[j] = in[j];
    a[j] = in[16 + j] + (float)threadIdx.x;
  }
  int ia = threadIdx.x, ib = (int)in[40];
  __syncthreads();
  long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
    if (VAR == 0) {
#pragma unroll
      for (int j = 0; j < 16; ++j) a[j] = __fadd_rn(a[j], b[j]);
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float2 r = __fadd2_rn(make_float2(a[2 * j], a[2 * j + 1]),
                              make_float2(b[2 * j], b[2 * j + 1]));
        a[2 * j] = r.x;
        a[2 * j + 1] = r.y;
        if (VAR == 2) ia = ia * 3 + ib;
      }
    }
  }
  __syncthreads();
  long long t1 = clock64();
  float sum = 0.0f;
#pragma unroll
  for (int j = 0; j < 16; ++j) sum += a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = sum + (float)ia;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

}  // namespace st

extern "C" st_status st_probe_add_rate(int32_t variant, int32_t iters, double* adds_per_clk_per_sm,
                                       double* tadds_per_s) {
  using namespace st;
  if (!adds_per_clk_per_sm || !tadds_per_s || variant < 0 || variant > 2 || iters <= 0)
    return ST_ERR_INVALID;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ST_ERR_CUDA;
  float* in = nullptr;
  float* out = nullptr;
  long long* cyc = nullptr;
  cudaEvent_t e0, e1;
  std::vector<float> h_in(48, 0.0f);
  for (int j = 0; j < 16; ++j) h_in[j] = 1e-7f * (j + 1);
  for (int j = 16; j < 32; ++j) h_in[j] = 0.5f * j;
  h_in[40] = 7.0f;
  if (cudaMalloc(&in, 48 * sizeof(float)) != cudaSuccess) return ST_ERR_OOM;
  cudaMalloc(&out, (size_t)sms * 1024 * sizeof(float));
  cudaMalloc(&cyc, (size_t)sms * sizeof(long long));
  cudaMemcpy(in, h_in.data(), 48 * sizeof(float), cudaMemcpyHostToDevice);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto run = [&](int it) {
    if (variant == 0) k_add_rate<0><<<sms, 1024>>>(in, out, it, cyc);
    else if (variant == 1) k_add_rate<1><<<sms, 1024>>>(in, out, it, cyc);
    else k_add_rate<2><<<sms, 1024>>>(in, out, it, cyc);
  };
  run(iters / 4 + 1);
  cudaEventRecord(e0);
  run(iters);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  std::vector<long long> h_cyc(sms);
  if (e == cudaSuccess) {
    cudaEventElapsedTime(&ms, e0, e1);
    e = cudaMemcpy(h_cyc.data(), cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
  }
  cudaFree(in);
  cudaFree(out);
  cudaFree(cyc);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return ST_ERR_CUDA;
  std::sort(h_cyc.begin(), h_cyc.end());
  double adds_per_block = 1024.0 * 16.0 * iters;
  *adds_per_clk_per_sm = adds_per_block / (double)h_cyc[sms / 2];
  *tadds_per_s = adds_per_block * sms / (ms * 1e-3) / 1e12;
  return ST_OK;
}

namespace st {
namespace {

// Waits on the first phase of an mbarrier that expects one arrival which
// never comes; the wait is bounded by limit_ns of the global timer.
__global__ void k_wait_probe(uint64_t limit_ns, int* timed_out, unsigned long long* waited_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_init_fence();
  const uint64_t t0 = global_ns();
  const bool ok = mbar_wait(&bar, 0u, limit_ns);
  *waited_ns = global_ns() - t0;
  *timed_out = ok ? 0 : 1;
}

}  // namespace
}  // namespace st

extern "C" st_status st_probe_wait_timeout(int32_t limit_us, int32_t* h_timed_out,
                                           double* h_waited_us) {
  using namespace st;
  if (!h_timed_out || !h_waited_us) return ST_ERR_INVALID;
  if (limit_us < 1 || limit_us > 2000000) return ST_ERR_INVALID;
  int* d_flag = nullptr;
  unsigned long long* d_ns = nullptr;
  if (cudaMalloc(&d_flag, sizeof(int)) != cudaSuccess) return ST_ERR_OOM;
  if (cudaMalloc(&d_ns, sizeof(unsigned long long)) != cudaSuccess) {
    cudaFree(d_flag);
    return ST_ERR_OOM;
  }
  k_wait_probe<<<1, 32>>>((uint64_t)limit_us * 1000ull, d_flag, d_ns);
  cudaError_t e = cudaDeviceSynchronize();
  int flag = 0;
  unsigned long long ns = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost);
  cudaFree(d_flag);
  cudaFree(d_ns);
  if (e != cudaSuccess) return ST_ERR_CUDA;
  *h_timed_out = flag;
  *h_waited_us = ns / 1000.0;
  return ST_OK;
}
