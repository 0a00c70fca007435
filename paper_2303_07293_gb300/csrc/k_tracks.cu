// k_tracks.cu — linking the per-velocity detections of one object into tracks.
//
// The search reports per-velocity local maxima (Sec. 2.1); a moving object
// yields detections at neighbouring trial velocities and positions, and the
// tracker reports tracks with speed, position angle, pixel coordinates and
// S/N.  Two detections of a field are linked when their pixels differ by at
// most r_xy in x and y and their velocity indices by at most r_v in a and b;
// a track is a connected component, represented by its detection of highest
// S/N (ties: the first in (field, k, y, x) order) with the component's size.
//
// The detections arrive sorted by (field, k, y, x), so a detection's
// neighbours at one (velocity, row) are a contiguous run found by binary
// search on the packed key.  Components come from a lock-free union-find
// (a root is hooked under the smaller root with a compare-and-swap, so every
// component's root is its first detection); tracks are listed in root order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <thrust/execution_policy.h>
#include <thrust/scan.h>

#include "st_internal.h"

namespace st {

namespace {

__device__ __forceinline__ uint64_t key_of(const st_candidate& c) {
  return cand_key(c.field, c.k, c.y, c.x);
}

// First index in [0, n) whose key is >= want.
__device__ int64_t lower_bound(const st_candidate* c, int64_t n, uint64_t want) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (key_of(c[mid]) < want) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ int find_root(int* parent, int x) {
  for (;;) {
    const int p = ((volatile int*)parent)[x];
    if (p == x) return x;
    const int gp = ((volatile int*)parent)[p];
    if (gp != p) ((volatile int*)parent)[x] = gp;  // path halving (stays inside the set)
    x = p;
  }
}

__device__ void unite(int* parent, int a, int b) {
  for (;;) {
    int ra = find_root(parent, a), rb = find_root(parent, b);
    if (ra == rb) return;
    if (ra > rb) {
      const int t = ra;
      ra = rb;
      rb = t;
    }
    // hook the larger root under the smaller one
    const int old = atomicCAS(&parent[rb], rb, ra);
    if (old == rb) return;
    b = old;  // rb gained a parent meanwhile: retry from there
    a = ra;
  }
}

__global__ void k_link_init(int* parent, unsigned long long* best, int* count, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  parent[i] = (int)i;
  best[i] = 0ull;
  count[i] = 0;
}

__global__ void k_link(const st_candidate* __restrict__ c, int64_t n,
                       const FieldDev* __restrict__ fds, int r_xy, int r_v, int* parent) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const st_candidate me = c[i];
  const FieldDev& fd = fds[me.field];
  const int a = me.k % fd.nvx, b = me.k / fd.nvx;
  for (int db = -r_v; db <= r_v; ++db) {
    const int b2 = b + db;
    if (b2 < 0 || b2 >= fd.nvy) continue;
    for (int da = -r_v; da <= r_v; ++da) {
      const int a2 = a + da;
      if (a2 < 0 || a2 >= fd.nvx) continue;
      const int k2 = b2 * fd.nvx + a2;
      for (int dy = -r_xy; dy <= r_xy; ++dy) {
        const int y2 = me.y + dy;
        if (y2 < 0 || y2 >= fd.H) continue;
        const int xlo = max(me.x - r_xy, 0), xhi = min(me.x + r_xy, fd.W - 1);
        const uint64_t khi = cand_key(me.field, k2, y2, xhi);
        for (int64_t j = lower_bound(c, n, cand_key(me.field, k2, y2, xlo));
             j < n && key_of(c[j]) <= khi; ++j)
          if (j > i) unite(parent, (int)i, (int)j);
      }
    }
  }
}

// Order-preserving map of an FP32 value to uint32 (larger float, larger key).
__device__ __forceinline__ uint32_t ordered(float v) {
  const uint32_t u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void k_link_reduce(const st_candidate* __restrict__ c, int64_t n, int* parent,
                              unsigned long long* best, int* count, int* is_root) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = find_root(parent, (int)i);
  // highest S/N, then the smallest index
  const unsigned long long key =
      ((unsigned long long)ordered(c[i].snr) << 32) | (0xffffffffu - (uint32_t)i);
  atomicMax(&best[r], key);
  atomicAdd(&count[r], 1);
  is_root[i] = r == (int)i ? 1 : 0;
}

__global__ void k_link_emit(const st_candidate* __restrict__ c, int64_t n,
                            const FieldDev* __restrict__ fds, const double* __restrict__ grid,
                            const int* is_root, const int* pos, const unsigned long long* best,
                            const int* count, st_track* __restrict__ out, int64_t cap) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !is_root[i] || pos[i] >= cap) return;
  const int64_t rep = 0xffffffffu - (uint32_t)(best[i] & 0xffffffffull);
  const st_candidate r = c[rep];
  const FieldDev& fd = fds[r.field];
  const double* g = grid + 4 * r.field;  // vx0, dvx, vy0, dvy
  const double vx = __dadd_rn(g[0], __dmul_rn((double)(r.k % fd.nvx), g[1]));
  const double vy = __dadd_rn(g[2], __dmul_rn((double)(r.k / fd.nvx), g[3]));
  double pa = atan2(-vx, -vy) * (180.0 / 3.14159265358979323846);
  if (pa < 0.0) pa += 360.0;
  st_track t;
  t.x = r.x;
  t.y = r.y;
  t.k = r.k;
  t.field = r.field;
  t.stack = r.stack;
  t.snr = r.snr;
  t.n_cov = r.n_cov;
  t.members = count[i];
  t.vx = (float)vx;
  t.vy = (float)vy;
  t.speed = (float)hypot(vx, vy);
  t.pa = (float)pa;
  out[pos[i]] = t;
}

}  // namespace

int64_t link_workspace_bytes(int64_t n) {
  return n * (int64_t)(sizeof(int) * 4 + sizeof(unsigned long long));
}

int launch_link_tracks(const st_candidate* c, int64_t n, const FieldDev* fds, const double* grid,
                       int r_xy, int r_v, void* ws, st_track* out, int64_t cap,
                       int64_t* n_tracks, cudaStream_t s) {
  *n_tracks = 0;
  if (n <= 0) return 0;
  unsigned long long* best = (unsigned long long*)ws;
  int* parent = (int*)(best + n);
  int* count = parent + n;
  int* is_root = count + n;
  int* pos = is_root + n;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  k_link_init<<<blocks, 256, 0, s>>>(parent, best, count, n);
  k_link<<<blocks, 256, 0, s>>>(c, n, fds, r_xy, r_v, parent);
  k_link_reduce<<<blocks, 256, 0, s>>>(c, n, parent, best, count, is_root);
  thrust::exclusive_scan(thrust::cuda::par.on(s), is_root, is_root + n, pos);
  k_link_emit<<<blocks, 256, 0, s>>>(c, n, fds, grid, is_root, pos, best, count, out, cap);
  int last_root = 0, last_pos = 0;
  cudaMemcpyAsync(&last_root, is_root + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&last_pos, pos + n - 1, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  *n_tracks = (int64_t)last_pos + last_root;
  return 5;
}

}  // namespace st
