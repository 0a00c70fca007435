// st_noalloc.cu — a search entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they search:
// processes whose device memory is fully reserved up front by another
// runtime or allocator, and hosts that forbid cudaMalloc after start-up
// (it can synchronise the device and take unbounded time).  st_stack_search_noalloc serves them: it runs the same kernels as
// st_stack_search for one field, but every scratch buffer it needs (shift
// tables, thresholds, counters, the above-threshold list, candidate records
// and sort keys) is carved out of one file-scope device array of
// kNoAllocScratchBytes.  The caller still provides the frames and the output
// buffer.
//
// The array is part of the library's device image: every GPU that loads the
// library holds it until the process exits.  Host code cannot use the array's
// symbol as a device address (on the host it names a stand-in object), so the
// first call on each device, with that device current, looks the address up
// with cudaGetSymbolAddress and caches it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "st_internal.h"

using namespace st;

namespace {

constexpr size_t kNoAllocScratchBytes = 32ull << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kMaxDevices] = {};

// Messages go to the storage behind st_last_error().
st_status na_fail(st_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return s;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device (looked up once).
st_status scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(ST_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(ST_ERR_UNSUPPORTED, "device id %d", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return na_fail(ST_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_noalloc_ptr[dev] = (unsigned char*)p;
  }
  *out = g_noalloc_ptr[dev];
  return ST_OK;
}

#define NA_CK(call)                                                                   \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return na_fail(ST_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

extern "C" st_status st_stack_search_noalloc(const st_field* field, int32_t mode,
                                             const float* d_frames, const double* h_times,
                                             st_candidate* d_out, int64_t capacity,
                                             int64_t* h_count, void* cuda_stream) {
  if (!field || !d_frames || !h_times || !h_count)
    return na_fail(ST_ERR_INVALID, "NULL argument");
  if (capacity < 0 || (capacity > 0 && !d_out))
    return na_fail(ST_ERR_INVALID, "capacity must be >= 0 and d_out non-NULL when capacity > 0");
  if (mode != ST_NEAREST && mode != ST_BILINEAR)
    return na_fail(ST_ERR_INVALID, "mode must be ST_NEAREST or ST_BILINEAR");
  const st_field& f = *field;
  if (f.width <= 0 || f.height <= 0 || f.width > 16384 || f.height > 16384 || f.n_frames <= 0 ||
      f.n_frames > 65535 || f.nvx <= 0 || f.nvy <= 0 || (int64_t)f.nvx * f.nvy > (1ll << 26) ||
      f.min_coverage < 0 || f.min_coverage > f.n_frames || !std::isfinite(f.snr_threshold) ||
      f.snr_threshold < 0.0f || !std::isfinite(f.t_ref) || !std::isfinite(f.vx0) ||
      !std::isfinite(f.dvx) || !std::isfinite(f.vy0) || !std::isfinite(f.dvy))
    return na_fail(ST_ERR_INVALID, "field out of range (same limits as st_plan)");
  double vmax = std::fmax(std::fmax(std::fabs(f.vx0), std::fabs(f.vx0 + (f.nvx - 1) * f.dvx)),
                          std::fmax(std::fabs(f.vy0), std::fabs(f.vy0 + (f.nvy - 1) * f.dvy)));
  for (int i = 0; i < f.n_frames; ++i) {
    if (!std::isfinite(h_times[i])) return na_fail(ST_ERR_INVALID, "timestamp %d not finite", i);
    if (vmax * std::fabs(h_times[i] - f.t_ref) > 1e9)
      return na_fail(ST_ERR_INVALID, "shift of frame %d exceeds 1e9 px", i);
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int N = f.n_frames;

  // Layout of the scratch array for this field.
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
  size_t o_ctr = take(sizeof(Counters));
  size_t o_fd = take(sizeof(FieldDev));
  size_t o_t = take(sizeof(double) * N);
  size_t o_sx = take(sizeof(int32_t) * (size_t)N * f.nvx);
  size_t o_sy = take(sizeof(int32_t) * (size_t)N * f.nvy);
  size_t o_fx = take(sizeof(float) * (size_t)N * f.nvx);
  size_t o_fy = take(sizeof(float) * (size_t)N * f.nvy);
  size_t o_thr = take(sizeof(float) * (N + 1));
  size_t o_rsq = take(sizeof(float) * (N + 1));
  if (off >= kNoAllocScratchBytes)
    return na_fail(ST_ERR_INVALID,
                   "tables of this field need %zu bytes, more than the %zu-byte no-alloc scratch",
                   off, kNoAllocScratchBytes);
  // above-threshold list, candidates and sort keys: 64 bytes per slot
  int64_t cap = 1;
  while ((size_t)(cap * 2) * 64 + off + 3 * 256 <= kNoAllocScratchBytes) cap *= 2;
  if (cap < 1024)
    return na_fail(ST_ERR_INVALID, "field leaves fewer than 1024 candidate slots in the %zu-byte "
                   "no-alloc scratch", kNoAllocScratchBytes);
  size_t o_pend = take(sizeof(Pending) * cap);
  size_t o_cand = take(sizeof(st_candidate) * cap);
  size_t o_keys = take(sizeof(uint64_t) * cap);
  size_t o_idx = take(sizeof(uint32_t) * cap);
  if (off > kNoAllocScratchBytes) return na_fail(ST_ERR_INVALID, "scratch layout overflow");

  unsigned char* base = nullptr;
  st_status st = scratch_address(&base);
  if (st != ST_OK) return st;
  Counters* ctr = (Counters*)(base + o_ctr);
  FieldDev* fdev = (FieldDev*)(base + o_fd);
  double* d_t = (double*)(base + o_t);
  int32_t* sx = (int32_t*)(base + o_sx);
  int32_t* sy = (int32_t*)(base + o_sy);
  float* fx = (float*)(base + o_fx);
  float* fy = (float*)(base + o_fy);
  float* thr = (float*)(base + o_thr);
  float* rsq = (float*)(base + o_rsq);
  Pending* pend = (Pending*)(base + o_pend);
  st_candidate* cand = (st_candidate*)(base + o_cand);
  uint64_t* keys = (uint64_t*)(base + o_keys);
  uint32_t* idx = (uint32_t*)(base + o_idx);

  // Threshold tables from the FP64 formulas, staged through a stack buffer
  // (pageable copies return once the source has been staged).
  float chunk[2][256];
  for (int n0 = 0; n0 <= N; n0 += 256) {
    int m = (N + 1 - n0) < 256 ? (N + 1 - n0) : 256;
    for (int j = 0; j < m; ++j) {
      int n = n0 + j;
      chunk[0][j] = (float)((double)f.snr_threshold * std::sqrt((double)n));
      chunk[1][j] = n > 0 ? (float)(1.0 / std::sqrt((double)n)) : 0.0f;
    }
    NA_CK(cudaMemcpyAsync(thr + n0, chunk[0], sizeof(float) * m, cudaMemcpyHostToDevice, s));
    NA_CK(cudaMemcpyAsync(rsq + n0, chunk[1], sizeof(float) * m, cudaMemcpyHostToDevice, s));
  }
  NA_CK(cudaMemcpyAsync(d_t, h_times, sizeof(double) * N, cudaMemcpyHostToDevice, s));
  launch_shift_tables(d_t, N, f.t_ref, f.vx0, f.dvx, f.nvx, f.vy0, f.dvy, f.nvy, mode, sx, sy, fx,
                      fy, s);
  FieldDev fd{};
  fd.cube = d_frames;
  fd.storage = ST_F32;
  fd.W = f.width;
  fd.H = f.height;
  fd.N = N;
  fd.nvx = f.nvx;
  fd.nvy = f.nvy;
  fd.nmin = f.min_coverage > 0 ? f.min_coverage : (N + 1) / 2;
  fd.field = 0;
  fd.sx = sx;
  fd.sy = sy;
  fd.fx = fx;
  fd.fy = fy;
  fd.thr = thr;
  fd.rsq = rsq;
  NA_CK(cudaMemcpyAsync(fdev, &fd, sizeof fd, cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), s));  // the previous call's counts remain
  launch_stack_generic(fd, mode, 0, f.nvx * f.nvy, nullptr, nullptr, nullptr, pend, cap, ctr, s);
  launch_resolve(fdev, 1, mode, pend, ctr, cap, cand, keys, idx, cap, ctr, s);
  NA_CK(cudaGetLastError());
  Counters hc;
  NA_CK(cudaMemcpyAsync(&hc, ctr, sizeof hc, cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (hc.error & ERR_PENDING_OVERFLOW) {
    *h_count = -1;
    return na_fail(ST_ERR_OVERFLOW, "%llu above-threshold points exceed the %lld slots of the "
                   "no-alloc scratch", (unsigned long long)hc.n_pending, (long long)cap);
  }
  int64_t n = (int64_t)hc.n_cand;
  int64_t sn = 1;
  while (sn < n) sn <<= 1;
  launch_pad_keys(keys, idx, sn, ctr, s);
  launch_sort_gather(keys, idx, sn, ctr, cand, d_out, capacity, s);
  NA_CK(cudaGetLastError());
  NA_CK(cudaStreamSynchronize(s));
  *h_count = n;
  if (n > capacity)
    return na_fail(ST_ERR_OVERFLOW, "%lld candidates exceed capacity %lld", (long long)n,
                   (long long)capacity);
  return ST_OK;
}
