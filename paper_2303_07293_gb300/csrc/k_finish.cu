// k_finish.cu — local-maximum test of the above-threshold points, candidate
// records, and the deterministic (field, k, y, x) ordering.
//
// Sec. 2.1 returns detections with pixel coordinates, motion and S/N.  The
// local-maximum rule (8 neighbours inside the frame with n_cov >= n_min;
// strictly greater than earlier neighbours in raster order, greater or equal
// to later ones) needs neighbour stack values that the stack kernels never
// store: they are recomputed here by the same ordered FP32 sum, so they are
// bit-identical to the values the stack kernel formed.
#include "st_internal.h"
#include "st_sample.cuh"

namespace st {

namespace {

template <typename T, int MODE>
__device__ void stack_one(const FieldDev& fd, int x, int y, int a, int b, float& S, int& C) {
  const T* cube = (const T*)fd.cube;
  const int64_t P = (int64_t)fd.W * fd.H;
  float acc = 0.0f;
  int cov = 0;
  for (int i = 0; i < fd.N; ++i) {
    const T* fr = cube + (int64_t)i * P;
    int u = x + __ldg(fd.sx + (int64_t)i * fd.nvx + a);
    int w = y + __ldg(fd.sy + (int64_t)i * fd.nvy + b);
    if (MODE == ST_NEAREST) {
      bool in = u >= 0 && w >= 0 && u < fd.W && w < fd.H;
      acc = __fadd_rn(acc, in ? load_px<T>(fr + (int64_t)w * fd.W + u) : 0.0f);
      cov += in;
    } else {
      float fx = __ldg(fd.fx + (int64_t)i * fd.nvx + a);
      float fy = __ldg(fd.fy + (int64_t)i * fd.nvy + b);
      BW wt = bilinear_weights(fx, fy);
      acc = bilinear_acc(acc, wt, tap<T>(fr, fd.W, fd.H, u, w), tap<T>(fr, fd.W, fd.H, u + 1, w),
                         tap<T>(fr, fd.W, fd.H, u, w + 1), tap<T>(fr, fd.W, fd.H, u + 1, w + 1));
      cov += bilinear_inside(u, fx, fd.W) && bilinear_inside(w, fy, fd.H);
    }
  }
  S = acc;
  C = cov;
}

template <int MODE>
__device__ void stack_any(const FieldDev& fd, int x, int y, int a, int b, float& S, int& C) {
  if (fd.storage == ST_F32) stack_one<float, MODE>(fd, x, y, a, b, S, C);
  else if (fd.storage == ST_F16) stack_one<__half, MODE>(fd, x, y, a, b, S, C);
  else stack_one<__nv_bfloat16, MODE>(fd, x, y, a, b, S, C);
}

// 8 threads per pending point (one per neighbour), 32 points per block.
template <int MODE>
__global__ void __launch_bounds__(256)
    k_resolve(const FieldDev* __restrict__ fds, const Pending* __restrict__ pend,
              const Counters* __restrict__ ctr_in, int64_t pend_cap,
              st_candidate* __restrict__ cand, uint64_t* __restrict__ keys,
              uint32_t* __restrict__ idx, int64_t cand_cap, Counters* __restrict__ ctr) {
  int64_t n = (int64_t)min((unsigned long long)pend_cap, ctr_in->n_pending);
  int64_t p = (int64_t)blockIdx.x * 32 + (threadIdx.x >> 3);
  int nb = threadIdx.x & 7;
  int lane = threadIdx.x & 31;
  bool have = p < n;
  Pending r{};
  bool q_in = false;
  float Sq = 0.0f;
  int Cq = 0;
  int nmin = 0;
  if (have) {
    r = pend[p];
    const FieldDev& fd = fds[r.field];
    nmin = fd.nmin;
    const int dxs[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
    const int dys[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
    int qx = r.x + dxs[nb], qy = r.y + dys[nb];
    if (qx >= 0 && qy >= 0 && qx < fd.W && qy < fd.H) {
      stack_any<MODE>(fd, qx, qy, r.k % fd.nvx, r.k / fd.nvx, Sq, Cq);
      q_in = true;
    }
    // a point recorded by position only: its own sum and coverage, same order
    if (nb == 0 && r.n_cov < 0) stack_any<MODE>(fd, r.x, r.y, r.k % fd.nvx, r.k / fd.nvx, r.S, r.n_cov);
  }
  const float Sc = __shfl_sync(0xffffffffu, r.S, lane & ~7);
  const int Cc = __shfl_sync(0xffffffffu, r.n_cov, lane & ~7);
  bool center_ok = false;
  if (have) center_ok = Cc >= nmin && Sc >= __ldg(fds[r.field].thr + Cc);
  const bool blocks = q_in && Cq >= nmin && (nb < 4 ? !(Sc > Sq) : !(Sc >= Sq));
  unsigned bal = __ballot_sync(0xffffffffu, blocks);
  unsigned group = (bal >> (lane & ~7)) & 0xffu;
  bool is_cand = center_ok && nb == 0 && group == 0u;
  unsigned m = __ballot_sync(0xffffffffu, is_cand);
  if (m == 0u) return;
  int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(&ctr->n_cand, (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (is_cand) {
    unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
    if (pos < (unsigned long long)cand_cap) {
      const FieldDev& fd = fds[r.field];
      st_candidate c;
      c.x = r.x;
      c.y = r.y;
      c.k = r.k;
      c.field = r.field;
      c.stack = r.S;
      c.snr = __fmul_rn(r.S, __ldg(fd.rsq + r.n_cov));
      c.n_cov = r.n_cov;
      cand[pos] = c;
      keys[pos] = cand_key(r.field, r.k, r.y, r.x);
      idx[pos] = (uint32_t)pos;
    } else {
      atomicOr(&ctr->error, ERR_CAND_OVERFLOW);
    }
  }
}

__global__ void k_pad_keys(uint64_t* keys, uint32_t* idx, int64_t n_pow2,
                           const Counters* __restrict__ ctr) {
  int64_t n = (int64_t)ctr->n_cand;
  int64_t i = n + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_pow2) {
    keys[i] = ~0ull;
    idx[i] = 0xffffffffu;
  }
}

__device__ __forceinline__ void cswap(uint64_t* keys, uint32_t* idx, int64_t i, int64_t l,
                                      bool asc) {
  uint64_t a = keys[i], b = keys[l];
  if ((a > b) == asc) {
    keys[i] = b;
    keys[l] = a;
    uint32_t t = idx[i];
    idx[i] = idx[l];
    idx[l] = t;
  }
}

__global__ void k_bitonic_global(uint64_t* keys, uint32_t* idx, int64_t n, int64_t j, int64_t k) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t l = i ^ j;
  if (l > i) cswap(keys, idx, i, l, (i & k) == 0);
}

constexpr int kLocal = 2048;  // elements per shared-memory tile

// All steps j < kLocal of stage k (k may be <= kLocal: then all stages up to k).
__global__ void __launch_bounds__(kLocal / 2)
    k_bitonic_local(uint64_t* keys, uint32_t* idx, int64_t n, int64_t k_from, int64_t k_to,
                    int64_t j_from) {
  __shared__ uint64_t sk[kLocal];
  __shared__ uint32_t si[kLocal];
  int64_t base = (int64_t)blockIdx.x * kLocal;
  for (int t = threadIdx.x; t < kLocal; t += blockDim.x) {
    sk[t] = base + t < n ? keys[base + t] : ~0ull;
    si[t] = base + t < n ? idx[base + t] : 0xffffffffu;
  }
  __syncthreads();
  for (int64_t k = k_from; k <= k_to; k <<= 1) {
    for (int64_t j = (k == k_from ? j_from : k >> 1); j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < kLocal; t += blockDim.x) {
        int l = t ^ (int)j;
        if (l > t) {
          bool asc = ((base + t) & k) == 0;
          uint64_t a = sk[t], b = sk[l];
          if ((a > b) == asc) {
            sk[t] = b;
            sk[l] = a;
            uint32_t q = si[t];
            si[t] = si[l];
            si[l] = q;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < kLocal; t += blockDim.x)
    if (base + t < n) {
      keys[base + t] = sk[t];
      idx[base + t] = si[t];
    }
}

__global__ void k_gather(const uint32_t* __restrict__ idx, const Counters* __restrict__ ctr,
                         const st_candidate* __restrict__ cand, st_candidate* __restrict__ out,
                         int64_t capacity) {
  int64_t n = min((int64_t)ctr->n_cand, capacity);
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) out[r] = cand[idx[r]];
}

}  // namespace

int launch_resolve(const FieldDev* fds_dev, int n_fields, int mode, const Pending* pend,
                   const Counters* ctr, int64_t pend_cap, st_candidate* cand, uint64_t* keys,
                   uint32_t* idx, int64_t cand_cap, Counters* ctr_out, cudaStream_t s) {
  (void)n_fields;
  // grid sized by the capacity; blocks past the live count exit at once
  int64_t blocks = (pend_cap + 31) / 32;
  if (mode == ST_NEAREST)
    k_resolve<ST_NEAREST><<<(unsigned)blocks, 256, 0, s>>>(fds_dev, pend, ctr, pend_cap, cand,
                                                           keys, idx, cand_cap, ctr_out);
  else
    k_resolve<ST_BILINEAR><<<(unsigned)blocks, 256, 0, s>>>(fds_dev, pend, ctr, pend_cap, cand,
                                                            keys, idx, cand_cap, ctr_out);
  return 1;
}

int launch_pad_keys(uint64_t* keys, uint32_t* idx, int64_t n_pow2, const Counters* ctr,
                    cudaStream_t s) {
  k_pad_keys<<<(unsigned)((n_pow2 + 255) / 256), 256, 0, s>>>(keys, idx, n_pow2, ctr);
  return 1;
}

int launch_sort_gather(uint64_t* keys, uint32_t* idx, int64_t n, const Counters* ctr,
                       const st_candidate* cand, st_candidate* out, int64_t capacity,
                       cudaStream_t s) {
  // n is a power of two >= the live count; padding keys sort last.
  int launches = 0;
  if (n >= 2) {
    int64_t tiles = (n + kLocal - 1) / kLocal;
    int64_t kmax_local = n < kLocal ? n : kLocal;
    k_bitonic_local<<<(unsigned)tiles, kLocal / 2, 0, s>>>(keys, idx, n, 2, kmax_local, 1);
    ++launches;
    for (int64_t k = 2 * kLocal; k <= n; k <<= 1) {
      for (int64_t j = k >> 1; j >= kLocal; j >>= 1) {
        k_bitonic_global<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, idx, n, j, k);
        ++launches;
      }
      k_bitonic_local<<<(unsigned)tiles, kLocal / 2, 0, s>>>(keys, idx, n, k, k, kLocal / 2);
      ++launches;
    }
  }
  if (capacity > 0) {
    int64_t g = (n < capacity ? n : capacity);
    if (g < 1) g = 1;
    k_gather<<<(unsigned)((g + 255) / 256), 256, 0, s>>>(idx, ctr, cand, out, capacity);
    ++launches;
  }
  return launches;
}

}  // namespace st
