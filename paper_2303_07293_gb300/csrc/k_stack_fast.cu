// k_stack_fast.cu — register-window shift-and-stack kernel for sm_103a.
//
// Computes the stack of the generic kernel (Sec. 1 / Sec. 2.1: every frame
// shifted by the trial motion v*(t_i - t_ref) and summed in frame order with
// one FP32 accumulator per output), laid out for the GB300 FP32 pipe, for
// nearest-pixel and bilinear sampling, over every field of a plan in one
// persistent launch:
//
// * A work item is a 32 x KY pixel tile (64 x KY for the column-pair
//   variant) of one field times a velocity tile of 8 x-velocities (one per
//   consumer warp) and 4 y-velocities (shared by all warps).  Lane l owns
//   column X0 + l (and X0 + 32 + l); each thread accumulates the KY rows of
//   its column for its warp's x-velocity and the 4 y-velocities.
// * A producer warp takes items from a work counter (fields longest first),
//   publishes each item in a shared-memory slot ring, and per frame issues a
//   TMA tile load of the item's footprint (zero-filled outside the frame)
//   into a ring of shared-memory stages guarded by mbarriers (full: bytes
//   landed; empty: all warps done), staging the frame's column offsets,
//   staircase pattern id (and bilinear fractions) beside it.  Every wait is
//   bounded.
// * A warp's x-shift is only an address: lane l reads column l + o_w, so the
//   32 lanes read 32 consecutive words (no bank conflicts, any alignment).
// * Each thread loads a window of its column (KY + 3 rows; bilinear: KY + 4
//   rows of the column and its right neighbour) and reuses every value for
//   the 4 y-velocities: y-velocity j reads window row r + c_j for output row
//   r.  The row offsets c_j form a monotone staircase with steps of 0 or 1
//   (15 patterns); the pattern is the same for the whole block in a frame, so
//   one switch per frame picks a straight-line body.  Accumulators are held
//   as row pairs (m, m + KY/2) and the window as pairs (q, q + KY/2), so
//   output pair m of y-velocity j adds window pair m + c_j: every add is a
//   paired add (add.f32x2) whatever the offsets' parity (the column-pair
//   variant pairs the two columns instead).  Bilinear: the warp's horizontal
//   interpolation of each window row is formed once and shared by the 4
//   y-velocities, each adding (1 - fy) h[r + c_j] + fy h[r + c_j + 1] as two
//   fused multiply-adds, paired the same way (fma.rn.f32x2).
// * After the last frame, outputs are compared with the item's lowest
//   possible threshold; the rare survivors go to the warp-aggregated pending
//   list, where the resolver forms their exact value, coverage and local
//   maximum with the generic kernel's arithmetic.
//
// Nearest sums are the same FP32 additions in the same order as the generic
// kernel (out-of-frame samples read +0.0 from the TMA zero fill), so the two
// kernels agree bit for bit; bilinear sums agree to FP32 rounding (the
// pre-filter keeps a margin for it).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <new>
#include <type_traits>
#include <utility>

#include "st_bodies.inc"
#include "st_internal.h"
#include "st_pending.cuh"
#include "st_sample.cuh"
#include "st_tma.cuh"

namespace st {

namespace {

constexpr int kXV = 8;           // x-velocities per block, one per warp (within a row group)
constexpr int kMB = 4;           // y-velocities per block (staircase group)
constexpr int kTX = 32;          // pixel tile width; its height is the variant's KY
// Storage traits: TMA box width (elements; 16-byte rows) and the largest
// column offset of a warp (16-bit storage: the 4-bit packing's limit).
template <typename T>
struct Store;
template <>
struct Store<float> {
  static constexpr int kBoxW = 40;
  static constexpr CUtensorMapDataType kTma = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  __device__ static float f(float v) { return v; }
};
template <>
struct Store<__half> {
  static constexpr int kBoxW = 48, kOColMax = 15;
  static constexpr CUtensorMapDataType kTma = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  __device__ static float f(__half v) { return __half2float(v); }
};
template <>
struct Store<__nv_bfloat16> {
  static constexpr int kBoxW = 48, kOColMax = 15;
  static constexpr CUtensorMapDataType kTma = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  __device__ static float f(__nv_bfloat16 v) { return __bfloat162float(v); }
};
constexpr int kSuper = 4;        // pixel tiles per super-tile side (L2 locality)
constexpr uint64_t kWaitNs = 2000000000ull;  // wait limit: 2 s of wall-clock time
constexpr unsigned kProducerSleepNs = 128;  // producer back-off between polls
constexpr int kPatterns = 15;
constexpr int kX2Wide = 8;       // extra box columns for 16 x-velocities a half
// table maxima: column offset in a tile, pattern id, shift spread, column
// offset in a pair of tiles
constexpr int kMaxes = 4;

// One field of a launch: geometry, per-frame tile tables and thresholds.
struct FastField {
  int W, H, N, nvx, nvy, nA, nB, nmin, field;
  const int4* xt;   // [N][nA]: box x offset, packed 4-bit column offsets, min shift, max shift
  const int4* yt;   // [N][nB]: min shift, max shift, pattern id, 0
  const unsigned char* pat;  // [N][nB] staircase pattern ids
  const int32_t* sx;
  const int32_t* sy;
  const float* fx;   // bilinear: FP32 fractions [N][nvx], [N][nvy]
  const float* fy;
  const float4* fxt;  // bilinear: [N][nA][2] x-fractions of a velocity tile's 8 x-velocities
  const float4* fyt;  // bilinear: [N][nB] y-fractions of its 4 y-velocities
  const float* thr;
  // coverage prefix tables: for velocity a, covx[a * cov_len + s - cov_xmin[a]]
  // = number of frames with sx(i, a) <= s (likewise y)
  const int* covx;
  const int* covy;
  const int* cov_xmin;
  const int* cov_xmax;
  const int* cov_ymin;
  const int* cov_ymax;
  int cov_len;
};

constexpr int kMaxFields = 256;

struct FastArgs {
  const FastField* ff[kMaxFields];    // the launch's fields, longest first (device)
  const CUtensorMap* maps[kMaxFields];  // their cubes' tiled maps (global memory)
  int n_fields;
  int64_t n_items;            // items of all fields
  unsigned long long* work;   // next item to take (zero at launch)
  Pending* pend;
  int64_t cap;
  Counters* ctr;
  float* dump_S;    // optional [nvx*nvy][H][W] of a single field (tests)
  int32_t* dump_C;
};

// Pattern id -> row offsets of the 4 y-velocities (min offset 0).
// ids 0..7: non-decreasing, steps (id&1, id>>1&1, id>>2&1);
// ids 8..14: non-increasing, steps of t = id - 7 read from the other end.
__host__ __device__ constexpr int pat_off(int id, int j) {
  if (id < 8) {
    int s1 = id & 1, s2 = (id >> 1) & 1, s3 = (id >> 2) & 1;
    return j == 0 ? 0 : j == 1 ? s1 : j == 2 ? s1 + s2 : s1 + s2 + s3;
  }
  int t = id - 7;
  int t1 = t & 1, t2 = (t >> 1) & 1, t3 = (t >> 2) & 1;
  return j == 0 ? t1 + t2 + t3 : j == 1 ? t2 + t3 : j == 2 ? t3 : 0;
}

__device__ int pattern_of(const int (&c)[kMB]) {
  for (int id = 0; id < kPatterns; ++id) {
    bool m = true;
    for (int j = 0; j < kMB; ++j) m = m && (pat_off(id, j) == c[j]);
    if (m) return id;
  }
  return 255;
}

__global__ void k_fast_tables(const int32_t* __restrict__ sx, const int32_t* __restrict__ sy,
                              int N, int nvx, int nvy, int nA, int nB, int4* __restrict__ xt,
                              int4* __restrict__ yt, int* xmin, int* xmax, int* ymin, int* ymax,
                              int* maxes, unsigned char* __restrict__ pat, int align) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t nX = (int64_t)N * nA, nY = (int64_t)N * nB;
  if (idx < nX) {
    int i = (int)(idx / nA), A = (int)(idx % nA);
    int s[kXV], mn = INT_MAX, mx = INT_MIN;
#pragma unroll
    for (int j = 0; j < kXV; ++j) {
      int a = min(A * kXV + j, nvx - 1);
      s[j] = sx[(int64_t)i * nvx + a];
      mn = min(mn, s[j]);
      mx = max(mx, s[j]);
    }
    int xs = mn & ~(align - 1);  // 16-byte aligned box origin (floor to a multiple of align)
    uint32_t packed = 0;
    int om = 0;
#pragma unroll
    for (int j = 0; j < kXV; ++j) {
      int o = s[j] - xs;
      om = max(om, o);
      packed |= (uint32_t)min(o, 15) << (4 * j);
    }
    xt[idx] = make_int4(xs, (int)packed, mn, mx);
    atomicMax(&maxes[0], om);
    if ((A & 1) == 0) {
      // tiles A and A + 1 as one box of 16 x-velocities (two a thread): its
      // largest column offset from the common aligned origin
      int mn16 = INT_MAX, mx16 = INT_MIN;
      for (int j = 0; j < 2 * kXV; ++j) {
        const int v = sx[(int64_t)i * nvx + min(A * kXV + j, nvx - 1)];
        mn16 = min(mn16, v);
        mx16 = max(mx16, v);
      }
      atomicMax(&maxes[3], mx16 - (mn16 & ~(align - 1)));
    }
    atomicMin(&xmin[A], mn);
    atomicMax(&xmax[A], mx);
  } else if (idx < nX + nY) {
    int64_t j2 = idx - nX;
    int i = (int)(j2 / nB), B = (int)(j2 % nB);
    int s[kMB], mn = INT_MAX, mx = INT_MIN;
#pragma unroll
    for (int j = 0; j < kMB; ++j) {
      int b = min(B * kMB + j, nvy - 1);
      s[j] = sy[(int64_t)i * nvy + b];
      mn = min(mn, s[j]);
      mx = max(mx, s[j]);
    }
    int c[kMB];
#pragma unroll
    for (int j = 0; j < kMB; ++j) c[j] = s[j] - mn;
    int id = pattern_of(c);
    yt[j2] = make_int4(mn, mx, id, 0);
    pat[j2] = (unsigned char)id;
    atomicMax(&maxes[1], id);
    atomicMin(&ymin[B], mn);
    atomicMax(&ymax[B], mx);
  }
}

// Largest spread of one velocity's shifts over the frames (one thread per velocity).
__global__ void k_shift_spread(const int32_t* __restrict__ sh, int N, int nv, int* out) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  int mn = INT_MAX, mx = INT_MIN;
  for (int i = 0; i < N; ++i) {
    int v = sh[(int64_t)i * nv + a];
    mn = min(mn, v);
    mx = max(mx, v);
  }
  atomicMax(out, mx - mn + 1);
}

// Coverage prefix tables of one axis: one thread per velocity.
__global__ void k_cov_tables(const int32_t* __restrict__ sh, int N, int nv, int len,
                             int* __restrict__ tab, int* __restrict__ vmin, int* __restrict__ vmax) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  int mn = INT_MAX, mx = INT_MIN;
  for (int i = 0; i < N; ++i) {
    int v = sh[(int64_t)i * nv + a];
    mn = min(mn, v);
    mx = max(mx, v);
  }
  vmin[a] = mn;
  vmax[a] = mx;
  int* row = tab + (int64_t)a * len;
  int span = mx - mn + 1;  // <= len (checked by the host)
  for (int s = 0; s < span; ++s) row[s] = 0;
  for (int i = 0; i < N; ++i) row[sh[(int64_t)i * nv + a] - mn] += 1;
  for (int s = 1; s < span; ++s) row[s] += row[s - 1];
}

// Row pairs: accumulator pair m of a y-velocity holds output rows m and
// m + KY/2, and pair window q holds window rows (q, q + KY/2).  Output row r
// of y-velocity j reads window row r + c_j, so pair m reads pair window
// m + c_j for any offset c_j: every add is a paired add (add.f32x2) on an
// aligned register pair, whatever the parity of the staircase offsets.
template <int KY, int C>
__device__ __forceinline__ void add_pair_column(float2 (&acc)[KY / 2],
                                                const float2 (&pw)[KY / 2 + 3]) {
#pragma unroll
  for (int m = 0; m < KY / 2; ++m) acc[m] = __fadd2_rn(acc[m], pw[m + C]);
}

template <int KY, int ID>
__device__ __forceinline__ void add_pattern(float2 (&acc)[kMB][KY / 2],
                                            const float2 (&pw)[KY / 2 + 3]) {
  add_pair_column<KY, pat_off(ID, 0)>(acc[0], pw);
  add_pair_column<KY, pat_off(ID, 1)>(acc[1], pw);
  add_pair_column<KY, pat_off(ID, 2)>(acc[2], pw);
  add_pair_column<KY, pat_off(ID, 3)>(acc[3], pw);
}

// Column pairs: the thread's two columns (c and c + 32) share every row
// offset, so window row r of both is one register pair and every add is a
// paired add: acc[j][r] += (wA[r + c_j], wB[r + c_j]).
template <int KY, int ID>
__device__ __forceinline__ void add_pattern_cp(float2 (&acc)[kMB][KY], const float2 (&w)[KY + 3]) {
#pragma unroll
  for (int j = 0; j < kMB; ++j)
#pragma unroll
    for (int r = 0; r < KY; ++r) acc[j][r] = __fadd2_rn(acc[j][r], w[r + pat_off(ID, j)]);
}

// Bilinear, factored: a warp's x-fraction is common to its 4 y-velocities, so
// the horizontal interpolation h[r] = c0[r] + fx (c1[r] - c0[r]) of window row
// r is formed once per frame and shared; y-velocity j then adds
// (1 - fy_j) h[r + c_j] + fy_j h[r + c_j + 1] to output row r as two fused
// multiply-adds, on row pairs (m, m + KY/2) as paired FMAs (fma.rn.f32x2)
// with the pair window hp[q] = (h[q], h[q + KY/2]).  (The generic kernel
// forms the same bilinear sample as four weighted taps; the two agree to
// FP32 rounding, and the local-maximum resolver re-forms every reported
// value with the generic arithmetic.)
template <int KY, int C>
__device__ __forceinline__ void add_bl_column(float2 (&acc)[KY / 2], float gy, float fy,
                                              const float2 (&hp)[KY / 2 + 4]) {
  const float2 g2 = make_float2(gy, gy), f2 = make_float2(fy, fy);
#pragma unroll
  for (int m = 0; m < KY / 2; ++m)
    acc[m] = __ffma2_rn(f2, hp[m + C + 1], __ffma2_rn(g2, hp[m + C], acc[m]));
}

template <int KY, int ID>
__device__ __forceinline__ void add_pattern_bl(float2 (&acc)[kMB][KY / 2], const float (&gy)[kMB],
                                               const float (&fy)[kMB],
                                               const float2 (&hp)[KY / 2 + 4]) {
  add_bl_column<KY, pat_off(ID, 0)>(acc[0], gy[0], fy[0], hp);
  add_bl_column<KY, pat_off(ID, 1)>(acc[1], gy[1], fy[1], hp);
  add_bl_column<KY, pat_off(ID, 2)>(acc[2], gy[2], fy[2], hp);
  add_bl_column<KY, pat_off(ID, 3)>(acc[3], gy[3], fy[3], hp);
}

// Number of frames whose shift s satisfies lo <= s <= hi, from a prefix table.
__device__ __forceinline__ int count_shifts(const int* pre, int smin, int smax, int N, int lo,
                                            int hi) {
  auto upto = [&](int s) { return s < smin ? 0 : s >= smax ? N : __ldg(pre + (s - smin)); };
  return hi < lo ? 0 : upto(hi) - upto(lo - 1);
}

__device__ int exact_coverage(const FastField& p, int x, int y, int av, int bv) {
  int c = 0;
  for (int i = 0; i < p.N; ++i) {
    int u = x + __ldg(p.sx + (int64_t)i * p.nvx + av);
    int w = y + __ldg(p.sy + (int64_t)i * p.nvy + bv);
    c += (u >= 0 && u < p.W && w >= 0 && w < p.H);
  }
  return c;
}

__device__ int exact_coverage_bl(const FastField& p, int x, int y, int av, int bv) {
  int c = 0;
  for (int i = 0; i < p.N; ++i) {
    int u = x + __ldg(p.sx + (int64_t)i * p.nvx + av);
    int w = y + __ldg(p.sy + (int64_t)i * p.nvy + bv);
    c += bilinear_inside(u, __ldg(p.fx + (int64_t)i * p.nvx + av), p.W) &&
         bilinear_inside(w, __ldg(p.fy + (int64_t)i * p.nvy + bv), p.H);
  }
  return c;
}

// Work item -> field, tile and velocity tile.  A field's items are ordered
// (super-tile, velocity tile, sub-tile) with the sub-tile fastest, so
// consecutive items (which neighbouring CTAs run at the same time) share most
// of their frame footprints in L2.  Fields are numbered longest first (most
// frames), so the short items of the last fields fill the tail.
struct Item {
  int f;           // index into the launch's field list (-1: no more work)
  int X0, Y0, A, B;
};
// Items of a field for tile height ky and width tx: super-tiles x 16 tiles x
// velocity tiles; an item of a CTA with h halves covers h x-velocity tiles
// (item A indexes groups of h tiles).
__device__ __host__ __forceinline__ int super_x_of(int W, int tx) {
  return ((W + tx - 1) / tx + kSuper - 1) / kSuper;
}
// tiles per super-tile column: 8-row tiles stack twice as many, so a
// super-tile covers the same pixels (and frame footprint in L2) as with
// 16-row tiles
__device__ __host__ __forceinline__ int super_h_of(int ky) { return ky == 8 ? 2 * kSuper : kSuper; }
__device__ __host__ __forceinline__ int groups_of(int nA, int h) { return (nA + h - 1) / h; }
__device__ __host__ __forceinline__ int64_t items_of(const FastField& ff, int ky, int tx,
                                                     int h) {
  const int sh = super_h_of(ky);
  const int sy = ((ff.H + ky - 1) / ky + sh - 1) / sh;
  return (int64_t)super_x_of(ff.W, tx) * sy * kSuper * sh * groups_of(ff.nA, h) * ff.nB;
}
__device__ __forceinline__ Item decode_item(const FastField& ff, int f, int64_t L, int ky,
                                            int tx, int h) {
  const int nAg = groups_of(ff.nA, h);
  const int nVT = nAg * ff.nB;
  const int super_x = super_x_of(ff.W, tx);
  const int sh = super_h_of(ky);
  const int sub = (int)(L % (kSuper * sh));
  const int64_t rest = L / (kSuper * sh);
  const int vt = (int)(rest % nVT);
  const int stile = (int)(rest / nVT);
  Item it;
  it.f = f;
  it.X0 = ((stile % super_x) * kSuper + sub % kSuper) * tx;
  it.Y0 = ((stile / super_x) * sh + sub / kSuper) * ky;
  it.A = vt % nAg;
  it.B = vt / nAg;
  return it;
}

// Acquire a tensor map written to global memory before the launch for the
// TMA unit (tensor-map proxy).
__device__ __forceinline__ void tmap_acquire(const CUtensorMap* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)m)
               : "memory");
}

// Persistent kernel over every item of every field of the launch (BL:
// bilinear sampling).  The last warp is the producer: it takes the next item from
// the launch's work counter (dynamic, in the fields' longest-first order),
// publishes the item in a ring of kItemSlots shared-memory slots, and runs
// ahead in stages of F frames (an item's frames are padded to whole stages
// with no-op frames, which have no copy): its lanes fetch the per-frame table
// entries, issue the TMA copies of a stage in parallel and publish the
// frames' column offsets, pattern ids (and bilinear fractions) and each
// item's count of fully-inside frames in shared memory.  The other 8 (or,
// with two halves, 16) warps consume.
// A ring of S stages runs continuously across items and fields; when the
// work runs out the producer publishes an end item.  Every wait is bounded.
// OPT (nearest sampling): bit 4 runs every stage of an item in one
// generated PTX block (st_bodies.inc): per frame, the warp's word(s) from
// the producer and an indexed branch into the pattern's body.  Otherwise a
// switch on the pattern id selects a C++ body.
// H: halves per CTA.  With H = 2 the CTA has 16 consumer warps and one
// producer (one CTA per SM, 96 registers a thread): an item covers two
// x-velocity tiles, each with its own box per frame and its own 8 warps.
// OPT bit 5 (KY = 8, with bit 4): two adjacent x-velocities a thread,
// so a half covers 16 x-velocities (two tables' tiles, one box 8 columns
// wider); on the frames where the two velocities' columns agree one window
// feeds both velocities' adds.
template <typename T, int KY, int S, int F, bool DUMP, bool BL, bool CP, int OPT, int H>
__device__ __forceinline__ void stack_fast_body(const FastArgs& p) {
  static_assert(!(CP && BL), "column pairs are built for nearest sampling");
  static_assert(H == 1 || !(CP || BL), "two halves are built for single-column nearest sampling");
  constexpr bool kX2 = (OPT & 32) != 0;
  constexpr int kXPW = kX2 ? 2 : 1;        // x-velocities per thread
  static_assert(!kX2 || ((OPT & 16) != 0 && KY == 8 && !BL && !CP),
                "two x-velocities a thread: nearest item loop, KY = 8");
  constexpr int kTXv = CP ? 2 * kTX : kTX;  // tile width: one or two columns per lane
  constexpr int kBoxW = Store<T>::kBoxW + (CP ? kTX : 0) + (kX2 ? kX2Wide : 0);
  constexpr int kAccN = CP ? KY : KY / 2;   // paired accumulators per y-velocity
  constexpr int kTY = KY;         // tile height: one row group of KY rows per thread
  constexpr int kBoxH = KY + 3 + (BL ? 1 : 0);  // tile rows + staircase offset (+ lower tap)
  constexpr int kEdge = BL ? 1 : 0;  // a bilinear sample also reads the next column / row
  constexpr int kCW = kXV * H;    // consumer warps
  constexpr int kOut = kMB * KY * (CP ? 2 : 1);  // outputs per thread and x-velocity
  constexpr int kItemSlots = 8;
  constexpr int kNoop = kPatterns;  // pattern id of a padding frame
  static_assert(F <= 4 || (OPT & 16) != 0, "pattern ids of a stage are packed into one word");
  extern __shared__ __align__(128) float smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[S];
  __shared__ __align__(8) uint64_t empty_bar[S];
  __shared__ __align__(16) uint32_t slot_ocol[S * H * F];  // packed 4-bit column offsets of 8 warps
  __shared__ uint32_t slot_ids[S];          // packed 8-bit pattern ids of the stage's frames
  // OPT bit 4: the whole item's stages (waits, frames, releases) in one PTX
  // block, fed per stage, warp and frame with the byte offset of the warp's
  // window in the ring and the pattern id in the top byte
  constexpr bool kItemPtx = (OPT & 16) != 0;
  constexpr bool kLean = kItemPtx;
  // (four words of padding: the PTX loop reads one frame's words ahead).
  // Two x-velocities a thread: four words per frame and warp (body index,
  // the two windows' byte offsets, one unused), read as one vector
  constexpr int kWords = kX2 ? 4 : 1;
  __shared__ __align__(16) uint32_t slot_word[kLean ? S * kCW * F * kWords + 4 : 1];
  __shared__ float slot_fx[BL ? S * F * kXV : 1];  // bilinear: x-fraction of each warp
  __shared__ float4 slot_fy[BL ? S * F : 1];       // bilinear: y-fractions of the 4 y-velocities
  __shared__ int item_inside[kItemSlots * H];  // frames of an item half fully inside the frame
  __shared__ int item_done[kItemSlots];     // consumer warps done with an item
  __shared__ Item item_info[kItemSlots];    // the items in flight

  T* smem = reinterpret_cast<T*>(reinterpret_cast<char*>(smem_raw) +
                                 ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t box_bytes = (uint32_t)kBoxH * kBoxW * sizeof(T);
  // one frame's box in elements, padded to 128 bytes (compile-time stride)
  constexpr int box_floats = ((kBoxH * kBoxW * (int)sizeof(T) + 127) & ~127) / (int)sizeof(T);

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], kCW);
    }
    mbar_init_fence();
  }
  if (tid < kItemSlots * H) item_inside[tid] = 0;
  if (tid < kItemSlots) item_done[tid] = 0;
  __syncthreads();

  if (warp == kCW) {
    // ------------------------------------------------------------ producer
    // Lane l < H*F handles frame l % F of a stage for half l / F.  The table
    // entries of the next stage are loaded while the current one waits for
    // its ring slot, and the next item's index is taken from the work counter
    // one item ahead, so neither global-memory latency sits between a free
    // slot and its copies.
    constexpr int kLanes = H * F;
    const int fi_l = lane % F, h_l = lane / F;
    int f = 0, acq_f = -1;
    int64_t base = 0;                                  // first item of field f
    int64_t f_items = items_of(*p.ff[0], KY, kTXv, H * kXPW);  // items of field f
    // the item of work-counter index L (-1: past the end); L only grows
    auto locate = [&](int64_t L) -> Item {
      Item it{-1, 0, 0, 0, 0};
      if (L >= p.n_items) return it;
      while (L >= base + f_items) {
        base += f_items;
        f_items = items_of(*p.ff[++f], KY, kTXv, H * kXPW);
      }
      return decode_item(*p.ff[f], f, L - base, KY, kTXv, H * kXPW);
    };
    auto take = [&]() -> int64_t {
      int64_t L = 0;
      if (lane == 0) L = (int64_t)atomicAdd(p.work, 1ull);
      return __shfl_sync(0xffffffffu, L, 0);
    };
    // the field of the current (and of the next) item, held in registers:
    // its descriptor in global memory is read once per field change
    struct Geo {
      int N, W, H, nA, nB;
      const int4* xt;
      const int4* yt;
      const unsigned char* pat;
      const float4* fxt;
      const float4* fyt;
    };
    auto geo_of = [&](int f) -> Geo {
      const FastField& ff = *p.ff[f];
      return Geo{ff.N, ff.W, ff.H, ff.nA, ff.nB, ff.xt, ff.yt, ff.pat, ff.fxt, ff.fyt};
    };
    // per-stage table entries of this lane's frame (valid: a real copy)
    struct Entry {
      int4 xe, ye;
      unsigned id;
      bool valid;
      float4 f0, f1, fy;
      // two x-velocities: the second tile's packed offsets, and both tiles'
      // box origins relative to the common box (bits 0..7 and 8..15)
      uint32_t oc1, dx;
    };
    auto load_entry = [&](const Item& it, const Geo& g, int st) -> Entry {
      Entry e{};
      e.id = kNoop;
      e.valid = false;
      if (it.f < 0 || lane >= kLanes) return e;
      const int fr = st * F + fi_l;
      const int A = it.A * H + h_l;
      if (fr >= g.N) return e;
      e.ye = __ldg(g.yt + (int64_t)fr * g.nB + it.B);
      e.id = g.pat[(int64_t)fr * g.nB + it.B];
      if constexpr (kX2) {
        // the half's 16 x-velocities: tiles 2A and 2A + 1 of the table (a
        // missing second tile repeats the first); one box from the lower
        // origin (both are multiples of 4 columns: 16-byte aligned)
        const int A0 = 2 * A, A1 = 2 * A + 1;
        if (A0 >= g.nA) return e;
        const int4 x0 = __ldg(g.xt + (int64_t)fr * g.nA + A0);
        const int4 x1 = A1 < g.nA ? __ldg(g.xt + (int64_t)fr * g.nA + A1) : x0;
        const int bx = min(x0.x, x1.x);
        e.xe = make_int4(bx, x0.y, min(x0.z, x1.z), max(x0.w, x1.w));
        e.oc1 = (uint32_t)x1.y;
        e.dx = (uint32_t)(x0.x - bx) | ((uint32_t)(x1.x - bx) << 8);
        e.valid = true;
        return e;
      }
      if (A >= g.nA) return e;  // the second half of a field's last tile group
      e.xe = __ldg(g.xt + (int64_t)fr * g.nA + A);
      e.valid = true;
      if constexpr (BL) {
        e.f0 = __ldg(g.fxt + 2 * ((int64_t)fr * g.nA + A));
        e.f1 = __ldg(g.fxt + 2 * ((int64_t)fr * g.nA + A) + 1);
        e.fy = __ldg(g.fyt + (int64_t)fr * g.nB + it.B);
      }
      return e;
    };
    int slot = 0;
    int64_t seq = 0;  // stages issued
    bool ok = true;
    Item it = locate(take());
    int64_t L_next = it.f >= 0 ? take() : p.n_items;
    int st = 0;
    Geo g = geo_of(it.f >= 0 ? it.f : 0);
    Entry cur = load_entry(it, g, 0);
    for (int item = 0; ok;) {
      const bool done = it.f < 0;
      const int N = done ? 1 : g.N;
      const int spi = (N + F - 1) / F;  // stages of this item (an end item: one)
      const CUtensorMap* map = done ? nullptr : p.maps[it.f];
      if (!done && it.f != acq_f) {
        if (lane == 0) {
          tmap_acquire(map);
          tma_prefetch_desc(map);
        }
        acq_f = it.f;
      }
      // the next stage: of this item, or the first of the next item
      Item it_n = it;
      Geo g_n = g;
      int st_n = st + 1;
      if (st_n == spi) {
        it_n = done ? it : locate(L_next);
        if (it_n.f >= 0 && it_n.f != it.f) g_n = geo_of(it_n.f);
        st_n = 0;
      }
      const Entry nxt = done ? cur : load_entry(it_n, g_n, st_n);
      if (seq >= S &&
          !mbar_wait_sleep(&empty_bar[slot], (uint32_t)(seq / S - 1) & 1u, kWaitNs,
                           kProducerSleepNs)) {
        if (lane == 0) atomicOr(&p.ctr->error, ERR_TIMEOUT);
        ok = false;
        break;  // consumers time out on the missing stage (bounded)
      }
      if (st == 0 && lane == 0) item_info[item % kItemSlots] = it;
      const unsigned copies = __ballot_sync(0xffffffffu, cur.valid);
      if (lane == 0 && copies) mbar_expect_tx(&full_bar[slot], box_bytes * __popc(copies));
      if constexpr (kX2) {
        // words (frame fi, warp w): the body index (the pattern id, plus 16
        // when the two columns differ; 15: no adds) and the ring offsets of
        // the windows of the thread's two x-velocities (16 x-velocities a
        // half, two a warp: 2 wl and 2 wl + 1, both of table tile wl / 4)
        const uint32_t oc0 = (uint32_t)cur.xe.y, oc1 = cur.oc1, dx = cur.dx;
        const uint32_t idv = cur.valid ? cur.id : (unsigned)kNoop;
#pragma unroll
        for (int k = lane; k < F * kCW; k += 32) {
          // lanes take consecutive word groups (frame fastest, as stored):
          // a warp's stores are conflict-free
          const int fi = k % F, w = k / F, h = w / kXV, wl = w % kXV;
          const int src = h * F + fi;
          const uint32_t a0 = __shfl_sync(0xffffffffu, oc0, src);
          const uint32_t a1 = __shfl_sync(0xffffffffu, oc1, src);
          const uint32_t d = __shfl_sync(0xffffffffu, dx, src);
          const uint32_t id = __shfl_sync(0xffffffffu, idv, src);
          const uint32_t pk = wl < kXV / 2 ? a0 : a1;            // the warp's table tile
          const uint32_t dg = wl < kXV / 2 ? d & 255u : d >> 8;  // its origin in the box
          const int i0 = (2 * wl) % kXV;
          const uint32_t o0 = dg + ((pk >> (4 * i0)) & 15u), o1 = dg + ((pk >> (4 * i0 + 4)) & 15u);
          const bool noop = id == (unsigned)kNoop;
          const uint32_t base = (uint32_t)(((slot * F + fi) * H + h) * box_floats * (int)sizeof(T));
          const uint32_t body = noop ? 15u : id + (o1 != o0 ? 16u : 0u);
          *reinterpret_cast<uint4*>(&slot_word[((slot * kCW + w) * F + fi) * 4]) =
              make_uint4(body, base + (noop ? 0u : o0) * (uint32_t)sizeof(T),
                         base + (noop ? 0u : o1) * (uint32_t)sizeof(T), 0u);
        }
      } else if constexpr (kLean) {
        // one word per lane: word (frame fi, warp w) of the stage, from the
        // entry of lane h * F + fi (its half's packed column offsets and id)
        const uint32_t ocw = (uint32_t)cur.xe.y;
        const uint32_t idv = cur.valid ? cur.id : (unsigned)kNoop;
#pragma unroll
        for (int k = lane; k < F * kCW; k += 32) {
          const int fi = k % F, w = k / F, h = w / kXV;  // consecutive words
          const uint32_t o = __shfl_sync(0xffffffffu, ocw, h * F + fi);
          const uint32_t id = __shfl_sync(0xffffffffu, idv, h * F + fi);
          const uint32_t oc = id == (unsigned)kNoop ? 0u : (o >> (4 * (w % kXV))) & 15u;
          const uint32_t base = (uint32_t)(((slot * F + fi) * H + h) * box_floats * (int)sizeof(T));
          slot_word[(slot * kCW + w) * F + fi] = (base + oc * (uint32_t)sizeof(T)) | (id << 24);
        }
      }
      if (cur.valid) {
        const int fr = st * F + fi_l;
        if constexpr (!kLean) slot_ocol[(slot * H + h_l) * F + fi_l] = (uint32_t)cur.xe.y;
        if constexpr (BL) {
          float* d = slot_fx + (slot * F + fi_l) * kXV;
          d[0] = cur.f0.x; d[1] = cur.f0.y; d[2] = cur.f0.z; d[3] = cur.f0.w;
          d[4] = cur.f1.x; d[5] = cur.f1.y; d[6] = cur.f1.z; d[7] = cur.f1.w;
          slot_fy[slot * F + fi_l] = cur.fy;
        }
        // every sample of the half strictly inside (bilinear: with its right
        // and lower taps), so every output of the half is covered
        const bool inside = it.X0 + cur.xe.z >= 0 &&
                            it.X0 + kTXv - 1 + cur.xe.w + kEdge < g.W &&
                            it.Y0 + cur.ye.x >= 0 && it.Y0 + kTY - 1 + cur.ye.y + kEdge < g.H;
        if (inside) atomicAdd(&item_inside[(item % kItemSlots) * H + h_l], 1);
        tma_load_3d(smem + (size_t)((slot * F + fi_l) * H + h_l) * box_floats, map,
                    it.X0 + cur.xe.x, it.Y0 + cur.ye.x, fr, &full_bar[slot]);
      }
      if constexpr (!kLean) {
        // the stage's ids (the same for both halves), packed: frame fi in byte fi
        uint32_t w = lane < F ? cur.id << (8 * lane) : 0u;
        w |= __shfl_xor_sync(0xffffffffu, w, 1);
        w |= __shfl_xor_sync(0xffffffffu, w, 2);
        if (lane == 0) slot_ids[slot] = w;
        __threadfence_block();
      }
      // the lanes' stores are ordered before lane 0's arrive (release) by the
      // warp barrier; consumers read them after their wait (acquire)
      __syncwarp();
      if (lane == 0) mbar_arrive(&full_bar[slot]);  // releases this stage's info
      if (++slot == S) slot = 0;
      ++seq;
      if (done) break;
      if (st_n == 0) {  // next item: take the one after it from the counter
        ++item;
        it = it_n;
        g = g_n;
        L_next = it.f >= 0 ? take() : p.n_items;
      }
      st = st_n;
      cur = nxt;
    }
    // drain (matters only after a consumer timeout): the last use of each
    // ring slot completes before the CTA may exit.  Only the latest phase of a
    // slot can be waited on: an older phase's parity aliases a newer one.
    if (lane == 0) {
      for (int64_t sq = seq > S ? seq - S : 0; sq < seq; ++sq)
        mbar_wait(&full_bar[sq % S], (uint32_t)(sq / S) & 1u, kWaitNs);
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  const int xw = warp % kXV, hw = warp / kXV;  // x-velocity in the half, half
  int c_slot = 0;
  uint32_t c_ph = 0;
  for (int item = 0;; ++item) {
    // the item's first stage carries its description
    if (!__all_sync(0xffffffffu, mbar_wait(&full_bar[c_slot], c_ph, kWaitNs))) {
      if (lane == 0) atomicOr(&p.ctr->error, ERR_TIMEOUT);  // leave (warp-uniform)
      break;
    }
    Item it = item_info[item % kItemSlots];
    if (it.f < 0) break;  // end of the work
    const FastField* ffp = p.ff[it.f];
    int N = ffp->N;
    const int spi = (N + F - 1) / F;
    float2 accx[kXPW][kMB][kAccN];
#pragma unroll
    for (int xx = 0; xx < kXPW; ++xx)
#pragma unroll
      for (int j = 0; j < kMB; ++j)
#pragma unroll
        for (int m = 0; m < kAccN; ++m) accx[xx][j][m] = make_float2(0.0f, 0.0f);
    float2 (&acc)[kMB][kAccN] = accx[0];
    // the accumulators as 64-bit register pairs for the PTX block (x-velocity
    // xx, y-velocity j, pair m: xx kMB kAccN + j kAccN + m)
    constexpr bool kAcc64 = kItemPtx;
    unsigned long long acc64[kAcc64 ? kXPW * kMB * kAccN : 1];
#pragma unroll
    for (int a = 0; a < (kAcc64 ? kXPW * kMB * kAccN : 1); ++a) acc64[a] = 0ull;

    bool ok = true;
    if constexpr (kItemPtx) {
      static_assert(KY == 16 || kX2, "the item loop is generated for KY = 16");
      constexpr bool kF32 = sizeof(T) == 4, kF16 = std::is_same<T, __half>::value;
      uint32_t slot = (uint32_t)c_slot, ph = c_ph, err = 0;
      __syncwarp();  // the item description is read before the block
      const uint32_t wb0 = smem_u32(&slot_word[warp * F * kWords]);
      const uint32_t lb = smem_u32(smem) + lane * (uint32_t)sizeof(T);
      const uint32_t fb0 = smem_u32(&full_bar[0]), eb0 = smem_u32(&empty_bar[0]);
      const uint32_t nst = (uint32_t)spi, skip = 1u;
#define ST_ITEM_ASM(NAME) \
  asm volatile(NAME ST_ITEM_OPERANDS_KY16(acc64, slot, ph, err, nst, skip, wb0, lb, fb0, eb0))
      // (two x-velocities of 8 rows: 32 accumulator pairs, as 16 rows of one)
      if constexpr (kX2 && !kF32 && F == 16 && S == 2 && kCW == 8 && kF16)
        ST_ITEM_ASM(ST_ITEMX2_KY8_F16_R112_S2_W8_F16);
      else if constexpr (kX2 && !kF32 && F == 16 && S == 2 && kCW == 8)
        ST_ITEM_ASM(ST_ITEMX2_KY8_F16_R112_S2_W8_BF16);
      else if constexpr (kX2 && !kF32)
        static_assert(F == 0, "no generated 16-bit two-velocity item loop for these stages and warps");
      else if constexpr (kX2 && F == 16 && S == 2 && kCW == 8)
        ST_ITEM_ASM(ST_ITEMX2_KY8_F16_R192_S2_W8);
      else if constexpr (kX2 && F == 16 && S == 2 && kCW == 16)
        ST_ITEM_ASM(ST_ITEMX2_KY8_F16_R192_S2_W16);
      else if constexpr (kX2)
        static_assert(F == 0, "no generated two-velocity item loop for these stages and warps");
      else if constexpr (!kF32 && F == 16 && S == 2 && kCW == 16 && kF16)
        ST_ITEM_ASM(ST_ITEM_KY16_F16_R96_S2_W16_F16);
      else if constexpr (!kF32 && F == 16 && S == 2 && kCW == 8 && kF16)
        ST_ITEM_ASM(ST_ITEM_KY16_F16_R96_S2_W8_F16);
      else if constexpr (!kF32 && F == 16 && S == 2 && kCW == 16)
        ST_ITEM_ASM(ST_ITEM_KY16_F16_R96_S2_W16_BF16);
      else if constexpr (!kF32 && F == 16 && S == 2 && kCW == 8)
        ST_ITEM_ASM(ST_ITEM_KY16_F16_R96_S2_W8_BF16);
      else if constexpr (!kF32)
        static_assert(F == 0, "no generated 16-bit item loop for these stages and warps");
      else if constexpr (F == 16 && S == 2 && kCW == 16)
        ST_ITEM_ASM(ST_ITEM_KY16_F16_R160_S2_W16);
      else if constexpr (F == 16 && S == 2 && kCW == 8)
        ST_ITEM_ASM(ST_ITEM_KY16_F16_R160_S2_W8);
      else if constexpr (F == 12 && S == 3 && kCW == 8)
        ST_ITEM_ASM(ST_ITEM_KY16_F12_R160_S3_W8);
      else if constexpr (F == 8 && S == 4 && kCW == 8)
        ST_ITEM_ASM(ST_ITEM_KY16_F8_R160_S4_W8);
      else if constexpr (F == 8 && S == 4 && kCW == 16)
        ST_ITEM_ASM(ST_ITEM_KY16_F8_R160_S4_W16);
      else
        static_assert(F == 0, "no generated item loop for these stages and warps");
#undef ST_ITEM_ASM
      c_slot = (int)slot;
      c_ph = ph;
      if (err) {
        if (lane == 0) atomicOr(&p.ctr->error, ERR_TIMEOUT);
        ok = false;
      }
      // read the item again (still in its slot: the producer is fewer than
      // kItemSlots items ahead), so nothing of it stays live across the block
      it = item_info[item % kItemSlots];
      ffp = p.ff[it.f];
      N = ffp->N;
    }
    const FastField& ff = *ffp;
    for (int st = 0; st < (kItemPtx ? 0 : spi); ++st) {
      if (st > 0 && !__all_sync(0xffffffffu, mbar_wait(&full_bar[c_slot], c_ph, kWaitNs))) {
        if (lane == 0) atomicOr(&p.ctr->error, ERR_TIMEOUT);
        ok = false;
        break;
      }
      const uint32_t idw = slot_ids[c_slot];  // the stage's pattern ids
      const T* stage = smem + (size_t)(c_slot * F * H + hw) * box_floats + lane;
      // this warp's column offsets of the stage's frames, 4 bits each, from
      // one vector load of the stage's packed words
      uint32_t ocw = 0;
      if constexpr (F == 4) {
        const uint4 q = *reinterpret_cast<const uint4*>(slot_ocol + (c_slot * H + hw) * F);
        ocw = ((q.x >> (4 * xw)) & 15u) | (((q.y >> (4 * xw)) & 15u) << 4) |
              (((q.z >> (4 * xw)) & 15u) << 8) | (((q.w >> (4 * xw)) & 15u) << 12);
      } else {
#pragma unroll
        for (int fi = 0; fi < F; ++fi)
          ocw |= ((slot_ocol[(c_slot * H + hw) * F + fi] >> (4 * xw)) & 15u) << (4 * fi);
      }
#pragma unroll 1
      for (int fi = 0; fi < F; ++fi) {
        const int id = (idw >> (8 * fi)) & 0xffu;
        const T* col = stage + fi * H * box_floats + ((ocw >> (4 * fi)) & 15u);
        if constexpr (BL) {
          float h[KY + 4];
          const float fxw = slot_fx[(c_slot * F + fi) * kXV + xw];
#pragma unroll
          for (int r = 0; r < KY + 4; ++r) {
            const float a0 = Store<T>::f(col[r * kBoxW]), a1 = Store<T>::f(col[r * kBoxW + 1]);
            h[r] = __fmaf_rn(fxw, __fsub_rn(a1, a0), a0);
          }
          float2 hp[KY / 2 + 4];
#pragma unroll
          for (int q = 0; q < KY / 2 + 4; ++q) hp[q] = make_float2(h[q], h[q + KY / 2]);
          const float4 fy4 = slot_fy[c_slot * F + fi];
          if (fi == F - 1) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty_bar[c_slot]);
          }
          const float fy[kMB] = {fy4.x, fy4.y, fy4.z, fy4.w};
          const float gy[kMB] = {__fsub_rn(1.0f, fy4.x), __fsub_rn(1.0f, fy4.y),
                                 __fsub_rn(1.0f, fy4.z), __fsub_rn(1.0f, fy4.w)};
          switch (id) {
            case 0: add_pattern_bl<KY, 0>(acc, gy, fy, hp); break;
            case 1: add_pattern_bl<KY, 1>(acc, gy, fy, hp); break;
            case 2: add_pattern_bl<KY, 2>(acc, gy, fy, hp); break;
            case 3: add_pattern_bl<KY, 3>(acc, gy, fy, hp); break;
            case 4: add_pattern_bl<KY, 4>(acc, gy, fy, hp); break;
            case 5: add_pattern_bl<KY, 5>(acc, gy, fy, hp); break;
            case 6: add_pattern_bl<KY, 6>(acc, gy, fy, hp); break;
            case 7: add_pattern_bl<KY, 7>(acc, gy, fy, hp); break;
            case 8: add_pattern_bl<KY, 8>(acc, gy, fy, hp); break;
            case 9: add_pattern_bl<KY, 9>(acc, gy, fy, hp); break;
            case 10: add_pattern_bl<KY, 10>(acc, gy, fy, hp); break;
            case 11: add_pattern_bl<KY, 11>(acc, gy, fy, hp); break;
            case 12: add_pattern_bl<KY, 12>(acc, gy, fy, hp); break;
            case 13: add_pattern_bl<KY, 13>(acc, gy, fy, hp); break;
            case 14: add_pattern_bl<KY, 14>(acc, gy, fy, hp); break;
            case kNoop: break;  // padding frame
            default: __builtin_unreachable();
          }
        } else if constexpr (CP) {
          float2 wp[KY + 3];  // rows of columns c and c + 32: register pairs
#pragma unroll
          for (int r = 0; r < KY + 3; ++r)
            wp[r] = make_float2(Store<T>::f(col[r * kBoxW]), Store<T>::f(col[r * kBoxW + kTX]));
          if (fi == F - 1) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty_bar[c_slot]);
          }
          switch (id) {
            case 0: add_pattern_cp<KY, 0>(acc, wp); break;
            case 1: add_pattern_cp<KY, 1>(acc, wp); break;
            case 2: add_pattern_cp<KY, 2>(acc, wp); break;
            case 3: add_pattern_cp<KY, 3>(acc, wp); break;
            case 4: add_pattern_cp<KY, 4>(acc, wp); break;
            case 5: add_pattern_cp<KY, 5>(acc, wp); break;
            case 6: add_pattern_cp<KY, 6>(acc, wp); break;
            case 7: add_pattern_cp<KY, 7>(acc, wp); break;
            case 8: add_pattern_cp<KY, 8>(acc, wp); break;
            case 9: add_pattern_cp<KY, 9>(acc, wp); break;
            case 10: add_pattern_cp<KY, 10>(acc, wp); break;
            case 11: add_pattern_cp<KY, 11>(acc, wp); break;
            case 12: add_pattern_cp<KY, 12>(acc, wp); break;
            case 13: add_pattern_cp<KY, 13>(acc, wp); break;
            case 14: add_pattern_cp<KY, 14>(acc, wp); break;
            case kNoop: break;  // padding frame
            default: __builtin_unreachable();
          }
        } else {
          float w[KY + 3];
#pragma unroll
          for (int r = 0; r < KY + 3; ++r) w[r] = Store<T>::f(col[r * kBoxW]);
          float2 pw[KY / 2 + 3];  // (row q, row q + KY/2) of the window
#pragma unroll
          for (int q = 0; q < KY / 2 + 3; ++q) pw[q] = make_float2(w[q], w[q + KY / 2]);
          if (fi == F - 1) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty_bar[c_slot]);
          }
          switch (id) {
            case 0: add_pattern<KY, 0>(acc, pw); break;
            case 1: add_pattern<KY, 1>(acc, pw); break;
            case 2: add_pattern<KY, 2>(acc, pw); break;
            case 3: add_pattern<KY, 3>(acc, pw); break;
            case 4: add_pattern<KY, 4>(acc, pw); break;
            case 5: add_pattern<KY, 5>(acc, pw); break;
            case 6: add_pattern<KY, 6>(acc, pw); break;
            case 7: add_pattern<KY, 7>(acc, pw); break;
            case 8: add_pattern<KY, 8>(acc, pw); break;
            case 9: add_pattern<KY, 9>(acc, pw); break;
            case 10: add_pattern<KY, 10>(acc, pw); break;
            case 11: add_pattern<KY, 11>(acc, pw); break;
            case 12: add_pattern<KY, 12>(acc, pw); break;
            case 13: add_pattern<KY, 13>(acc, pw); break;
            case 14: add_pattern<KY, 14>(acc, pw); break;
            case kNoop: break;  // padding frame
            default: __builtin_unreachable();
          }
        }
      }
      if (++c_slot == S) {
        c_slot = 0;
        c_ph ^= 1u;
      }
    }
    if (!ok) break;
    if constexpr (kAcc64) {
#pragma unroll
      for (int xx = 0; xx < kXPW; ++xx)
#pragma unroll
        for (int j = 0; j < kMB; ++j)
#pragma unroll
          for (int m = 0; m < kAccN; ++m)
            asm("mov.b64 {%0, %1}, %2;" : "=f"(accx[xx][j][m].x), "=f"(accx[xx][j][m].y)
                : "l"(acc64[(xx * kMB + j) * kAccN + m]));
    }

    // ---- epilogue of the item (its last stage was waited on, so the
    // producer's count is visible)
    const int n_full = item_inside[(item % kItemSlots) * H + hw];
    const int x = it.X0 + lane;
#pragma unroll
    for (int xx = 0; xx < kXPW; ++xx) {
    float2 (&acc)[kMB][kAccN] = accx[xx];
    // the thread's x-velocity: x-velocity tile (it.A H + hw) of kXV kXPW
    const int av = ((it.A * H + hw) * kXV + xw) * kXPW + xx;
    if constexpr (CP) {
      // outputs (j, r, h): y-velocity j, row r, column x + 32 h; value
      // acc[j][r].x (h = 0) or .y (h = 1); bit o = (j KY + r) 2 + h
      if constexpr (DUMP) {
#pragma unroll
        for (int j = 0; j < kMB; ++j)
#pragma unroll
          for (int r = 0; r < KY; ++r)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int bv = it.B * kMB + j, y = it.Y0 + r, xh = x + kTX * h;
              if (xh < ff.W && y < ff.H && av < ff.nvx && bv < ff.nvy) {
                const int64_t o =
                    ((int64_t)bv * ff.nvx + av) * ff.W * (int64_t)ff.H + (int64_t)y * ff.W + xh;
                p.dump_S[o] = h == 0 ? acc[j][r].x : acc[j][r].y;
                if (p.dump_C) p.dump_C[o] = exact_coverage(ff, xh, y, av, bv);
              }
            }
      } else {
        constexpr int kWords = (kOut + 31) / 32;
        uint32_t mask[kWords];
#pragma unroll
        for (int b = 0; b < kWords; ++b) mask[b] = 0u;
        const bool ok0 = x < ff.W && av < ff.nvx, ok1 = x + kTX < ff.W && av < ff.nvx;
        if (n_full == N) {
          const float thr_n = __ldg(ff.thr + max(N, ff.nmin));
#pragma unroll
          for (int j = 0; j < kMB; ++j)
#pragma unroll
            for (int r = 0; r < KY; ++r) {
              const int o = (j * KY + r) * 2;
              mask[o / 32] |= (uint32_t)(ok0 && acc[j][r].x >= thr_n) << (o % 32);
              mask[o / 32] |= (uint32_t)(ok1 && acc[j][r].y >= thr_n) << (o % 32 + 1);
            }
        } else {
          // edge item: as for single columns, with nx per column
          const int avc = min(av, ff.nvx - 1);
          const int* px = ff.covx + (int64_t)avc * ff.cov_len;
          const int sxmin = __ldg(ff.cov_xmin + avc), sxmax = __ldg(ff.cov_xmax + avc);
          const int nx0 = count_shifts(px, sxmin, sxmax, N, -x, ff.W - 1 - kEdge - x);
          const int nx1 =
              count_shifts(px, sxmin, sxmax, N, -(x + kTX), ff.W - 1 - kEdge - (x + kTX));
#pragma unroll
          for (int j = 0; j < kMB; ++j) {
            const int bvc = min(it.B * kMB + j, ff.nvy - 1);
            const int y = it.Y0 + lane % KY;
            int ny = count_shifts(ff.covy + (int64_t)bvc * ff.cov_len, __ldg(ff.cov_ymin + bvc),
                                  __ldg(ff.cov_ymax + bvc), N, -y, ff.H - 1 - kEdge - y);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) ny = min(ny, __shfl_xor_sync(0xffffffffu, ny, d));
            const int base = max(n_full, ff.nmin);
            const float thr0 = __ldg(ff.thr + min(max(base, nx0 + ny - N), N));
            const float thr1 = __ldg(ff.thr + min(max(base, nx1 + ny - N), N));
#pragma unroll
            for (int r = 0; r < KY; ++r) {
              const int o = (j * KY + r) * 2;
              mask[o / 32] |= (uint32_t)(ok0 && acc[j][r].x >= thr0) << (o % 32);
              mask[o / 32] |= (uint32_t)(ok1 && acc[j][r].y >= thr1) << (o % 32 + 1);
            }
          }
        }
        for (int b = 0; b < kWords; ++b) {
          uint32_t mk = mask[b];
          while (__any_sync(0xffffffffu, mk != 0u)) {
            const bool has = mk != 0u;
            const int bit = has ? __ffs(mk) - 1 : 0;
            mk &= has ? mk - 1u : 0u;
            const int o = b * 32 + bit;
            const int j = o / (2 * KY), y = it.Y0 + (o >> 1) % KY, bv = it.B * kMB + j;
            const int xh = x + kTX * (o & 1);
            const bool valid = has && y < ff.H && bv < ff.nvy;
            Pending rec{xh, y, bv * ff.nvx + av, ff.field, 0.0f, -1};
            push_pending(valid, rec, p.pend, p.cap, p.ctr);
          }
        }
      }
    } else {
      if constexpr (DUMP) {
  #pragma unroll
        for (int j = 0; j < kMB; ++j)
  #pragma unroll
          for (int m = 0; m < KY / 2; ++m)
  #pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int bv = it.B * kMB + j, y = it.Y0 + m + h * (KY / 2);
              if (x < ff.W && y < ff.H && av < ff.nvx && bv < ff.nvy) {
                const int64_t o =
                    ((int64_t)bv * ff.nvx + av) * ff.W * (int64_t)ff.H + (int64_t)y * ff.W + x;
                p.dump_S[o] = h == 0 ? acc[j][m].x : acc[j][m].y;
                if (p.dump_C)
                  p.dump_C[o] = BL ? exact_coverage_bl(ff, x, y, av, bv)
                                   : exact_coverage(ff, x, y, av, bv);
              }
            }
      } else {
        // outputs at or above the block's lowest possible threshold, as a
        // bitmask; the exact coverage, threshold and local-maximum test of
        // these rare points happen in the resolver
        constexpr int kWords = (kOut + 31) / 32;
        uint32_t mask[kWords];
  #pragma unroll
        for (int b = 0; b < kWords; ++b) mask[b] = 0u;
        // bilinear: the resolver re-forms each value with the generic
        // arithmetic, which differs from the factored form by FP32 rounding;
        // the pre-filter threshold is lowered by a relative 2e-4 of the
        // threshold's scale so no point is dropped for that reason
        auto lower = [&](float t) {
          return BL ? t - 2e-4f * (fabsf(t) + sqrtf((float)N)) : t;
        };
        if (n_full == N) {
          // interior item: every output is covered by all N frames
          const float thr_n = lower(__ldg(ff.thr + max(N, ff.nmin)));
  #pragma unroll
          for (int j = 0; j < kMB; ++j)
  #pragma unroll
            for (int m = 0; m < KY / 2; ++m) {
              const int o0 = j * KY + m, o1 = o0 + KY / 2;  // rows m and m + KY/2
              mask[o0 / 32] |= (uint32_t)(acc[j][m].x >= thr_n) << (o0 % 32);
              mask[o1 / 32] |= (uint32_t)(acc[j][m].y >= thr_n) << (o1 % 32);
            }
        } else {
          // edge item: n_cov >= nx + ny - N, with nx / ny the frames whose x / y
          // sample is inside (bilinear: with its right / lower tap, which
          // implies inside for any fraction; ny taken at the item's least
          // covered row), and n_cov >= n_full; thresholds grow with n_cov, so
          // this never drops a candidate
          const int avc = min(av, ff.nvx - 1);
          const int nx = count_shifts(ff.covx + (int64_t)avc * ff.cov_len,
                                      __ldg(ff.cov_xmin + avc), __ldg(ff.cov_xmax + avc), N, -x,
                                      ff.W - 1 - kEdge - x);
  #pragma unroll
          for (int j = 0; j < kMB; ++j) {
            // ny minimised over the item's rows (lane l takes row l % KY)
            const int bvc = min(it.B * kMB + j, ff.nvy - 1);
            const int y = it.Y0 + lane % KY;
            int ny = count_shifts(ff.covy + (int64_t)bvc * ff.cov_len, __ldg(ff.cov_ymin + bvc),
                                  __ldg(ff.cov_ymax + bvc), N, -y, ff.H - 1 - kEdge - y);
  #pragma unroll
            for (int d = 16; d > 0; d >>= 1) ny = min(ny, __shfl_xor_sync(0xffffffffu, ny, d));
            const int nlo = max(max(n_full, ff.nmin), nx + ny - N);
            const float thr_j = lower(__ldg(ff.thr + min(nlo, N)));
  #pragma unroll
            for (int m = 0; m < KY / 2; ++m) {
              const int o0 = j * KY + m, o1 = o0 + KY / 2;  // rows m and m + KY/2
              mask[o0 / 32] |= (uint32_t)(acc[j][m].x >= thr_j) << (o0 % 32);
              mask[o1 / 32] |= (uint32_t)(acc[j][m].y >= thr_j) << (o1 % 32);
            }
          }
        }
        const bool col_ok = x < ff.W && av < ff.nvx;
        for (int b = 0; b < kWords; ++b) {
          uint32_t mk = col_ok ? mask[b] : 0u;
          while (__any_sync(0xffffffffu, mk != 0u)) {
            const bool has = mk != 0u;
            const int bit = has ? __ffs(mk) - 1 : 0;
            mk &= has ? mk - 1u : 0u;
            const int o = b * 32 + bit;
            const int j = o / KY, y = it.Y0 + o % KY, bv = it.B * kMB + j;
            const bool valid = has && y < ff.H && bv < ff.nvy;
            Pending rec{x, y, bv * ff.nvx + av, ff.field, 0.0f, -1};
            push_pending(valid, rec, p.pend, p.cap, p.ctr);
          }
        }
      }
    }
    }  // x-velocities of the thread
    // release the item's count slot: the last warp to finish the item clears
    // it (the producer is at most S stages, fewer than kItemSlots - 1 items,
    // ahead of the slowest warp)
    __syncwarp();
    if (lane == 0 && atomicAdd(&item_done[item % kItemSlots], 1) == kCW - 1) {
#pragma unroll
      for (int h = 0; h < H; ++h) item_inside[(item % kItemSlots) * H + h] = 0;
      item_done[item % kItemSlots] = 0;
    }
  }
}

// Kernels: one CTA of 9 warps (two per SM for KY <= 16), or, with two
// halves, one CTA of 17 warps per SM; either way 96 registers a thread (the
// 5 warps of the fullest SM sub-partition share its 16 K registers).
template <typename T, int KY, int S, int F, bool DUMP, bool BL, bool CP, int OPT, int H>
__global__ void __launch_bounds__(32 * (kXV + 1), KY <= 16 ? 2 : 1)
    k_stack_fast(const __grid_constant__ FastArgs p) {
  stack_fast_body<T, KY, S, F, DUMP, BL, CP, OPT, 1>(p);
}
template <typename T, int KY, int S, int F, bool DUMP, bool BL, bool CP, int OPT, int H>
__global__ void __launch_bounds__(32 * (2 * kXV + 1), 1) k_stack_fast_h2(const __grid_constant__ FastArgs p) {
  stack_fast_body<T, KY, S, F, DUMP, BL, CP, OPT, 2>(p);
}

template <typename T, int KY, int S, int F, bool DUMP, bool BL, bool CP, int OPT, int H>
constexpr void (*kernel_of())(FastArgs) {
  if constexpr (H == 1)
    return k_stack_fast<T, KY, S, F, DUMP, BL, CP, OPT, 1>;
  else
    return k_stack_fast_h2<T, KY, S, F, DUMP, BL, CP, OPT, 2>;
}

// Compiled variants: (rows per thread, stages, frames per stage), each with
// and without the stack dump used by the tests.
struct Variant {
  void (*fn)(FastArgs);
  void (*dump_fn)(FastArgs);
  int threads, stages, ky, stages_f;
  int tx;  // tile width: 32 (one column per lane) or 64 (column pairs)
  int halves;  // x-velocity tiles per item (boxes per frame)
  int xpw;     // x-velocities per thread (2: a half holds two table tiles)
  const char* name;
};

#define ST_VARIANT(T, KY, S, F, BL, CP, OPT, H)                                               \
  {                                                                                           \
    kernel_of<T, KY, S, F, false, BL, CP, OPT, H>(),                                          \
        kernel_of<T, KY, S, F, true, BL, CP, OPT, H>(),                                       \
        32 * (kXV * H + 1), S * F, KY, F, CP ? 2 * kTX : kTX, H, (OPT & 32) ? 2 : 1,           \
        #T "_ky" #KY "_s" #S "_f" #F "_cp" #CP "_o" #OPT "_h" #H                                \
  }
#define NEAR(T, KY, S, F) ST_VARIANT(T, KY, S, F, false, false, 0, 1)
// the whole item's stages in one PTX block, pattern bodies that load the
// window rows as they add them (FP32, KY = 16); ITEMH: two x-velocity tiles
// per item, one CTA of 16 consumer warps and a producer per SM
#define ITEM(T, KY, S, F) ST_VARIANT(T, KY, S, F, false, false, 16, 1)
#define ITEMH(T, KY, S, F) ST_VARIANT(T, KY, S, F, false, false, 16, 2)
// two adjacent x-velocities a thread (FP32, KY = 8): one window feeds both
// velocities' adds on the frames where their columns agree
#define ITEMX(T, KY, S, F) ST_VARIANT(T, KY, S, F, false, false, 48, 1)
#define ITEMXH(T, KY, S, F) ST_VARIANT(T, KY, S, F, false, false, 48, 2)
#define PAIR(T, KY, S, F) ST_VARIANT(T, KY, S, F, false, true, 0, 1)
#define BILI(T, KY, S, F) ST_VARIANT(T, KY, S, F, true, false, 0, 1)
// (the first is the default; a two-velocity variant whose boxes do not hold
// a field's motion runs as the first single-velocity one)
const Variant kVarF32[] = {ITEMX(float, 8, 2, 16), ITEMH(float, 16, 2, 16), ITEM(float, 16, 2, 16),
                           ITEM(float, 16, 3, 12), ITEM(float, 16, 4, 8), ITEMH(float, 16, 4, 8),
                           NEAR(float, 16, 8, 4), NEAR(float, 24, 6, 4), PAIR(float, 8, 8, 4),
                           ITEMXH(float, 8, 2, 16)};
const Variant kVarF16[] = {ITEMX(__half, 8, 2, 16), ITEMH(__half, 16, 2, 16),
                           ITEM(__half, 16, 2, 16), NEAR(__half, 16, 8, 4), PAIR(__half, 8, 8, 4)};
const Variant kVarBF16[] = {ITEMX(__nv_bfloat16, 8, 2, 16), ITEMH(__nv_bfloat16, 16, 2, 16),
                            ITEM(__nv_bfloat16, 16, 2, 16), NEAR(__nv_bfloat16, 16, 8, 4),
                            PAIR(__nv_bfloat16, 8, 8, 4)};
// bilinear sampling: two window columns, one shared horizontal interpolation
const Variant kVarBlF32[] = {BILI(float, 8, 8, 4), BILI(float, 12, 8, 4), BILI(float, 16, 6, 4)};
const Variant kVarBlF16[] = {BILI(__half, 8, 8, 4), BILI(__half, 12, 8, 4)};
const Variant kVarBlBF16[] = {BILI(__nv_bfloat16, 8, 8, 4), BILI(__nv_bfloat16, 12, 8, 4)};
#undef NEAR
#undef ITEM
#undef ITEMH
#undef ITEMX
#undef ITEMXH
#undef PAIR
#undef BILI
#undef ST_VARIANT
constexpr int kNumVariants = sizeof(kVarF32) / sizeof(kVarF32[0]);  // the largest list

#define ST_LIST(L)                            \
  {                                           \
    *count = (int)(sizeof(L) / sizeof(L[0])); \
    return L;                                 \
  }
const Variant* variants_for(int storage, bool bl, int* count) {
  if (bl) {
    if (storage == ST_F16) ST_LIST(kVarBlF16);
    if (storage == ST_BF16) ST_LIST(kVarBlBF16);
    ST_LIST(kVarBlF32);
  }
  if (storage == ST_F16) ST_LIST(kVarF16);
  if (storage == ST_BF16) ST_LIST(kVarBF16);
  ST_LIST(kVarF32);
}
#undef ST_LIST

// The variant that runs in place of a two-velocity one whose boxes do not
// hold the motion: the first single-velocity one of the list.
int single_velocity_fallback(const Variant* vars, int n) {
  for (int v = 0; v < n; ++v)
    if (vars[v].xpw == 1) return v;
  return 0;
}

// TMA box width of a variant (elements)
int box_w_of(const Variant& v, int storage) {
  return (storage == ST_F32 ? Store<float>::kBoxW : Store<__half>::kBoxW) + (v.tx - kTX) +
         (v.xpw > 1 ? kX2Wide : 0);
}

// Fractions of a velocity tile, gathered per frame: fxt[(i nA + A) 8 + w] =
// fx(i, 8A + w) and fyt[(i nB + B) 4 + j] = fy(i, 4B + j) (clamped to the grid).
__global__ void k_frac_tables(const float* __restrict__ fx, const float* __restrict__ fy, int N,
                              int nvx, int nvy, int nA, int nB, float* __restrict__ fxt,
                              float* __restrict__ fyt) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t nX = (int64_t)N * nA * kXV, nY = (int64_t)N * nB * kMB;
  if (idx < nX) {
    int64_t i = idx / (nA * kXV);
    int a = (int)(idx % (nA * kXV));
    fxt[idx] = fx[i * nvx + min(a, nvx - 1)];
  } else if (idx < nX + nY) {
    idx -= nX;
    int64_t i = idx / (nB * kMB);
    int b = (int)(idx % (nB * kMB));
    fyt[idx] = fy[i * nvy + min(b, nvy - 1)];
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

}  // namespace

struct FastPlan {
  CUtensorMap tmap;
  const void* encoded_for = nullptr;
  int encoded_boxh = 0;
  int encoded_boxw = 0;
  int variant = 0;         // index into the (storage type, sampling) variant list
  bool bl = false;         // bilinear sampling
  int64_t item_limit = 0;  // > 0: run only the first item_limit items (autotuning)
  int nA = 0, nB = 0, N = 0;
  unsigned char* d_pat = nullptr;  // [N][nB] pattern ids
  FastField h_ff{};                // the field's descriptor (host copy)
  FastField* d_ff = nullptr;       // and on the device
  CUtensorMap* d_map = nullptr;    // the cube's tiled map on the device (64-byte aligned)
  int4* xt = nullptr;
  int4* yt = nullptr;
  float* fxt = nullptr;   // bilinear: [N][nA][8] x-fractions
  float* fyt = nullptr;   // bilinear: [N][nB][4] y-fractions
  int* ranges = nullptr;  // xmin[nA], xmax[nA], ymin[nB], ymax[nB], maxes[kMaxes]
  int* h_maxes = nullptr; // pinned
  bool fits_x2 = false;   // the two-velocity variants' wider boxes hold the motion
  int* cov = nullptr;     // covx [nvx*len], covy [nvy*len], mins/maxes [2*nvx + 2*nvy]
  int cov_len = 0;
  int64_t cov_cap = 0;
};

int fast_plan_size_bytes() { return (int)sizeof(FastPlan); }

bool encode_tile_map(CUtensorMap* map, const FieldDev& fd, int box_w, int box_h) {
  if (!encode_fn()) return false;
  const int esz = fd.storage == ST_F32 ? 4 : 2;
  const CUtensorMapDataType dtype = fd.storage == ST_F32    ? Store<float>::kTma
                                    : fd.storage == ST_F16 ? Store<__half>::kTma
                                                           : Store<__nv_bfloat16>::kTma;
  if (((int64_t)fd.W * esz) % 16 != 0) return false;  // row pitch: a multiple of 16 bytes
  cuuint64_t dims[3] = {(cuuint64_t)fd.W, (cuuint64_t)fd.H, (cuuint64_t)fd.N};
  cuuint64_t strides[2] = {(cuuint64_t)fd.W * esz, (cuuint64_t)fd.W * fd.H * esz};
  cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return encode_fn()(map, dtype, 3, const_cast<void*>(fd.cube), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int fast_num_variants() { return kNumVariants; }

int fast_num_variants_for(const FastPlan* fp, int storage) {
  int n = 0;
  variants_for(storage, fp && fp->bl, &n);
  return n;
}

int fast_get_variant(const FastPlan* fp) { return fp ? fp->variant : -1; }

// Times the register-window variants on the first `items` work items and
// keeps the fastest.  Pushes to the pending list (callers reset counters).
int fast_autotune(const FieldDev& fd, FastPlan* fp, int64_t items, Pending* pend,
                  int64_t pend_cap, Counters* ctr, cudaStream_t s) {
  int n = 0;
  const Variant* vars = variants_for(fd.storage, fp->bl, &n);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int best_v = fp->variant;
  int launches = 0;
  fp->item_limit = items;
  for (int v = 0; v < n; ++v) {
    if (vars[v].xpw > 1 && !fp->fits_x2) continue;  // its boxes do not hold the motion
    fp->variant = v;
    float ms_min = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {  // first run warms up
      cudaEventRecord(e0, s);
      int l = launch_stack_fast(fd, fp, 0, fd.nvx * fd.nvy, nullptr, nullptr, nullptr, pend,
                                pend_cap, ctr, s);
      cudaEventRecord(e1, s);
      if (l < 0 || cudaEventSynchronize(e1) != cudaSuccess) break;
      launches += l;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < ms_min) ms_min = ms;
    }
    if (ms_min < best) {
      best = ms_min;
      best_v = v;
    }
  }
  fp->item_limit = 0;
  fp->variant = best_v;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return launches;
}
const char* fast_variant_name(const FastPlan* fp, int storage) {
  int n = 0;
  const Variant* vars = variants_for(storage, fp && fp->bl, &n);
  int v = fp ? fp->variant : -1;
  if (v >= 0 && v < n && vars[v].xpw > 1 && !fp->fits_x2)
    v = single_velocity_fallback(vars, n);  // as the launch runs it
  return v >= 0 && v < n ? vars[v].name : "?";
}
void fast_set_variant(FastPlan* fp, int v) {
  if (fp && v >= 0 && v < kNumVariants) fp->variant = v;
}

bool fast_eligible(const FieldDev& fd, int mode) {
  const int align = fd.storage == ST_F32 ? 4 : 8;  // 16-byte rows for the tensor map
  return (mode == ST_NEAREST || mode == ST_BILINEAR) && fd.W % align == 0 &&
         encode_fn() != nullptr && fd.W >= 8 && fd.H >= 1;
}

bool fast_plan_build(const FieldDev& fd, int mode, FastPlan** out) {
  *out = nullptr;
  FastPlan* fp = new (std::nothrow) FastPlan();
  if (!fp) return false;
  fp->nA = (fd.nvx + kXV - 1) / kXV;
  fp->nB = (fd.nvy + kMB - 1) / kMB;
  fp->N = fd.N;
  fp->bl = mode == ST_BILINEAR;
  const size_t nfx = fp->bl ? (size_t)fd.N * fp->nA * kXV : 1;
  const size_t nfy = fp->bl ? (size_t)fd.N * fp->nB * kMB : 1;
  bool good = cudaMalloc(&fp->fxt, sizeof(float) * nfx) == cudaSuccess &&
              cudaMalloc(&fp->fyt, sizeof(float) * nfy) == cudaSuccess &&
              cudaMalloc(&fp->xt, sizeof(int4) * (size_t)fd.N * fp->nA) == cudaSuccess &&
              cudaMalloc(&fp->yt, sizeof(int4) * (size_t)fd.N * fp->nB) == cudaSuccess &&
              cudaMalloc(&fp->ranges, sizeof(int) * (2 * fp->nA + 2 * fp->nB + kMaxes)) == cudaSuccess &&
              cudaMallocHost(&fp->h_maxes, sizeof(int) * kMaxes) == cudaSuccess &&
              cudaMalloc(&fp->d_pat, (size_t)fd.N * fp->nB) == cudaSuccess &&
              cudaMalloc(&fp->d_ff, sizeof(FastField)) == cudaSuccess &&
              cudaMalloc(&fp->d_map, sizeof(CUtensorMap)) == cudaSuccess;
  if (!good) {
    fast_plan_free(fp);
    return false;
  }
  *out = fp;
  return true;
}

void fast_plan_free(FastPlan* fp) {
  if (!fp) return;
  cudaFree(fp->xt);
  cudaFree(fp->yt);
  cudaFree(fp->fxt);
  cudaFree(fp->fyt);
  cudaFree(fp->ranges);
  cudaFree(fp->cov);
  if (fp->h_maxes) cudaFreeHost(fp->h_maxes);
  cudaFree(fp->d_pat);
  cudaFree(fp->d_ff);
  cudaFree(fp->d_map);
  delete fp;
}

// Builds the per-frame tile tables and reports whether the field's motion
// fits the kernel (column offsets within the box, 8 for FP32 nearest, 7 for
// FP32 bilinear, 15 for 16-bit storage, among 8 x-velocities; staircase row
// offsets within 4 y-velocities).  Synchronises s.
int fast_prepare(const FieldDev& fd, FastPlan* fp, cudaStream_t s, bool* fits) {
  *fits = false;
  int nA = fp->nA, nB = fp->nB;
  int* xmin = fp->ranges;
  int* xmax = xmin + nA;
  int* ymin = xmax + nA;
  int* ymax = ymin + nB;
  int* maxes = ymax + nB;
  cudaMemsetAsync(xmin, 0x7f, sizeof(int) * nA, s);
  cudaMemsetAsync(xmax, 0x80, sizeof(int) * nA, s);
  cudaMemsetAsync(ymin, 0x7f, sizeof(int) * nB, s);
  cudaMemsetAsync(ymax, 0x80, sizeof(int) * nB, s);
  cudaMemsetAsync(maxes, 0, sizeof(int) * kMaxes, s);
  int64_t n = (int64_t)fd.N * (nA + nB);
  k_fast_tables<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(fd.sx, fd.sy, fd.N, fd.nvx, fd.nvy, nA,
                                                            nB, fp->xt, fp->yt, xmin, xmax, ymin,
                                                            ymax, maxes, fp->d_pat,
                                                            fd.storage == ST_F32 ? 4 : 8);
  if (fp->bl) {
    int64_t nf = (int64_t)fd.N * (nA * kXV + nB * kMB);
    k_frac_tables<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(fd.fx, fd.fy, fd.N, fd.nvx, fd.nvy,
                                                               nA, nB, fp->fxt, fp->fyt);
  }
  k_shift_spread<<<(fd.nvx + 127) / 128, 128, 0, s>>>(fd.sx, fd.N, fd.nvx, maxes + 2);
  k_shift_spread<<<(fd.nvy + 127) / 128, 128, 0, s>>>(fd.sy, fd.N, fd.nvy, maxes + 2);
  cudaMemcpyAsync(fp->h_maxes, maxes, sizeof(int) * kMaxes, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return 1;
  // coverage prefix tables: one row per velocity, as long as the widest spread
  const int len = fp->h_maxes[2];
  const int64_t need = (int64_t)(fd.nvx + fd.nvy) * (len + 2);
  if (len <= 0 || need > (64ll << 20)) return 1;  // tables too large: generic kernel
  if (need > fp->cov_cap) {
    cudaFree(fp->cov);
    fp->cov = nullptr;
    fp->cov_cap = 0;
    if (cudaMalloc(&fp->cov, sizeof(int) * need) != cudaSuccess) return 1;
    fp->cov_cap = need;
  }
  fp->cov_len = len;
  int* covx = fp->cov;
  int* covy = covx + (int64_t)fd.nvx * len;
  int* cxmin = covy + (int64_t)fd.nvy * len;
  int* cxmax = cxmin + fd.nvx;
  int* cymin = cxmax + fd.nvx;
  int* cymax = cymin + fd.nvy;
  k_cov_tables<<<(fd.nvx + 127) / 128, 128, 0, s>>>(fd.sx, fd.N, fd.nvx, len, covx, cxmin, cxmax);
  k_cov_tables<<<(fd.nvy + 127) / 128, 128, 0, s>>>(fd.sy, fd.N, fd.nvy, len, covy, cymin, cymax);
  if (cudaGetLastError() != cudaSuccess) return 1;
  // the field's descriptor for the kernel (pageable source: the copy is
  // staged before cudaMemcpyAsync returns)
  FastField& h = fp->h_ff;
  h = FastField{};
  h.W = fd.W;
  h.H = fd.H;
  h.N = fd.N;
  h.nvx = fd.nvx;
  h.nvy = fd.nvy;
  h.nA = nA;
  h.nB = nB;
  h.nmin = fd.nmin;
  h.field = fd.field;
  h.xt = fp->xt;
  h.yt = fp->yt;
  h.pat = fp->d_pat;
  h.sx = fd.sx;
  h.sy = fd.sy;
  h.fx = fd.fx;
  h.fy = fd.fy;
  h.fxt = reinterpret_cast<const float4*>(fp->fxt);
  h.fyt = reinterpret_cast<const float4*>(fp->fyt);
  h.thr = fd.thr;
  h.cov_len = len;
  h.covx = covx;
  h.covy = covy;
  h.cov_xmin = cxmin;
  h.cov_xmax = cxmax;
  h.cov_ymin = cymin;
  h.cov_ymax = cymax;
  if (cudaMemcpyAsync(fp->d_ff, &h, sizeof(FastField), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return 1;
  // N >= 8 (two stages of 4 frames): the producer runs at most S stages (at
  // most 48 frames) ahead of the slowest consumer, so fewer than 8 items are
  // live and the 8 per-item slots never collide.  Bilinear reads one more
  // column: lane 31 + ocol + 1 must stay in the box.
  const int ocol_max = fd.storage == ST_F32
                           ? Store<float>::kBoxW - kTX - (fp->bl ? 1 : 0)
                           : Store<__half>::kOColMax;
  *fits = fp->h_maxes[0] <= ocol_max && fp->h_maxes[1] < kPatterns && fd.N >= 8;
  // two x-velocities a thread: lane 31 + the column offset within the
  // wider box
  const int box_w = fd.storage == ST_F32 ? Store<float>::kBoxW : Store<__half>::kBoxW;
  fp->fits_x2 = *fits && !fp->bl && fp->h_maxes[3] <= box_w + kX2Wide - kTX;
  return 1;
}

// The launch's variant (that of fps[0]) and, for every field, its cube's
// tiled map for that variant's box, encoded and copied to the device when the
// cube or the box changed (pageable source: staged before the call returns).
static const Variant* stage_maps(const FieldDev* fds, FastPlan* const* fps, int n,
                                 cudaStream_t s, bool* restaged, int* vi_out) {
  if (n < 1 || n > kMaxFields) return nullptr;
  FastPlan* fp0 = fps[0];
  int nvar = 0;
  const Variant* vars = variants_for(fds[0].storage, fp0->bl, &nvar);
  int vi = fp0->variant < nvar ? fp0->variant : 0;
  // a two-velocity variant needs every field's motion within its boxes
  for (int i = 0; i < n && vars[vi].xpw > 1; ++i)
    if (!fps[i]->fits_x2) vi = single_velocity_fallback(vars, nvar);
  const Variant& var = vars[vi];
  const int boxh = var.ky + 3 + (fp0->bl ? 1 : 0);
  const int boxw = box_w_of(var, fds[0].storage);
  for (int i = 0; i < n; ++i) {
    FastPlan* fp = fps[i];
    if (fds[i].storage != fds[0].storage || fp->bl != fp0->bl) return nullptr;
    if (fp->encoded_for != fds[i].cube || fp->encoded_boxh != boxh ||
        fp->encoded_boxw != boxw) {
      if (!encode_tile_map(&fp->tmap, fds[i], boxw, boxh)) return nullptr;
      if (cudaMemcpyAsync(fp->d_map, &fp->tmap, sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                          s) != cudaSuccess)
        return nullptr;
      fp->encoded_for = fds[i].cube;
      fp->encoded_boxh = boxh;
      fp->encoded_boxw = boxw;
      if (restaged) *restaged = true;
    }
  }
  // kernel attributes are set once per compiled kernel
  static bool attr_set[2][3][2 * kNumVariants] = {};
  for (int d = 0; d < 2; ++d)
    if (!attr_set[fp0->bl][fds[0].storage][2 * vi + d]) {
      // as much dynamic shared memory as the device allows beside the
      // kernel's static shared memory
      const void* fn = (const void*)(d ? var.dump_fn : var.fn);
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      cudaFuncAttributes fa{};
      cudaFuncGetAttributes(&fa, fn);
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes);
      attr_set[fp0->bl][fds[0].storage][2 * vi + d] = true;
    }
  *vi_out = vi;
  return &var;
}

bool fast_stage(const FieldDev* fds, FastPlan* const* fps, int n, cudaStream_t s,
                bool* restaged) {
  int vi = 0;
  return stage_maps(fds, fps, n, s, restaged, &vi) != nullptr;
}

int launch_stack_fast_multi(const FieldDev* fds, FastPlan* const* fps, int n, float* dump_S,
                            int32_t* dump_C, Pending* pend, int64_t pend_cap, Counters* ctr,
                            cudaStream_t s) {
  FastPlan* fp0 = fps[0];  // the variant of the launch
  int vi = 0;
  const Variant* vp = stage_maps(fds, fps, n, s, nullptr, &vi);
  if (!vp) return -1;
  const Variant& var = *vp;
  const int ky = var.ky, boxh = ky + 3 + (fp0->bl ? 1 : 0);
  const int boxw = box_w_of(var, fds[0].storage);
  // fields longest first (the items of the most frames are taken first)
  int order[kMaxFields];
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order, order + n, [&](int x, int y) { return fds[x].N > fds[y].N; });
  thread_local static FastArgs a;
  std::memset(&a, 0, sizeof a);
  int64_t total = 0;
  for (int i = 0; i < n; ++i) {
    a.ff[i] = fps[order[i]]->d_ff;
    a.maps[i] = fps[order[i]]->d_map;
    total += items_of(fps[order[i]]->h_ff, ky, var.tx, var.halves * var.xpw);
  }
  a.n_fields = n;
  // an autotuning run covers the same work for every variant: item_limit
  // items of 32 x 16 pixels and 8 x-velocities
  const int64_t unit = (int64_t)var.halves * var.xpw * var.ky * var.tx;  // per 8 x-velocities
  const int64_t limit = fp0->item_limit > 0 ? (fp0->item_limit * 16 * kTX + unit - 1) / unit : 0;
  a.n_items = limit > 0 && total > limit ? limit : total;
  a.work = &ctr->work_next;
  a.pend = pend;
  a.cap = pend_cap;
  a.ctr = ctr;
  a.dump_S = dump_S;
  a.dump_C = dump_C;
  const int esz = fds[0].storage == ST_F32 ? 4 : 2;
  const int stage_bytes = ((boxh * boxw * esz) + 127) & ~127;
  void (*fn)(FastArgs) = dump_S ? var.dump_fn : var.fn;
  const size_t smem = (size_t)var.stages * var.halves * stage_bytes + 128;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMemsetAsync(&ctr->work_next, 0, sizeof(ctr->work_next), s) != cudaSuccess) return -1;
  // persistent CTAs per SM: as many as are resident at once (2 for KY <= 16),
  // queried once per compiled kernel
  static int resident[2][3][2 * kNumVariants] = {};
  int& per_sm = resident[fp0->bl][fds[0].storage][2 * vi + (dump_S ? 1 : 0)];
  if (per_sm < 1 &&
      (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn, var.threads,
                                                     smem) != cudaSuccess ||
       per_sm < 1))
    per_sm = 1;
  const int64_t grid = a.n_items < (int64_t)sms * per_sm ? a.n_items : (int64_t)sms * per_sm;
  if (grid < 1) return 0;
  void* args[1] = {&a};
  if (cudaLaunchKernel((const void*)fn, dim3((unsigned)grid), dim3(var.threads), args, smem, s) !=
      cudaSuccess)
    return -1;
  return 1;
}

int launch_stack_fast(const FieldDev& fd, const FastPlan* cfp, int k0, int nk,
                      const int32_t* dump_k, float* dump_S, int32_t* dump_C, Pending* pend,
                      int64_t pend_cap, Counters* ctr, cudaStream_t s) {
  if (k0 != 0 || nk != fd.nvx * fd.nvy || dump_k) return -1;  // whole grid only
  FastPlan* fp = const_cast<FastPlan*>(cfp);
  return launch_stack_fast_multi(&fd, &fp, 1, dump_S, dump_C, pend, pend_cap, ctr, s);
}

}  // namespace st
