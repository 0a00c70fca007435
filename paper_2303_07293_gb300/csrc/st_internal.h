// st_internal.h — internal types of the synthetic-tracking library (device +
// host).  Not part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/st.h"

namespace st {

// Above-threshold point waiting for the local-maximum test (24 bytes).
struct Pending {
  int32_t x, y, k, field;
  float S;
  int32_t n_cov;
};

// Counters shared by the kernels of one search, in device memory.
struct Counters {
  unsigned long long n_pending;   // points written (or attempted) to the pending list
  unsigned long long n_cand;      // candidates after the local-maximum test
  unsigned int error;             // bit flags, ERR_*
  unsigned int pad;
  unsigned long long work_next;   // persistent-kernel work counter
};

enum : unsigned { ERR_PENDING_OVERFLOW = 1u, ERR_CAND_OVERFLOW = 2u, ERR_TIMEOUT = 4u };

// Everything a kernel needs to read one field.  Plain data, passed by value.
struct FieldDev {
  const void* cube;      // storage cube [N][H][W] of `storage` type
  int32_t storage;       // st_dtype
  int32_t W, H, N;
  int32_t nvx, nvy;
  int32_t nmin;
  int32_t field;
  const int32_t* sx;     // [N][nvx] integer shift (nearest: rounded; bilinear: floor)
  const int32_t* sy;     // [N][nvy]
  const float* fx;       // [N][nvx] bilinear fraction
  const float* fy;       // [N][nvy]
  const float* thr;      // [N+1] thr[n] = (float)(tau*sqrt(n))
  const float* rsq;      // [N+1] (float)(1/sqrt(n))
};

// Key of a candidate: (field, k, y, x) packed into 64 bits, increasing in
// the output order.
__host__ __device__ inline uint64_t cand_key(int field, int k, int y, int x) {
  return ((uint64_t)(uint32_t)field << 56) | ((uint64_t)(uint32_t)k << 30) |
         ((uint64_t)(uint32_t)y << 15) | (uint64_t)(uint32_t)x;
}

// Sets the message returned by st_last_error() on this thread.
void set_last_error(const char* msg);

// ---- kernel launchers (each returns the number of kernels it launched) ----

int launch_shift_tables(const double* d_t, int N, double t_ref, double vx0, double dvx,
                        int nvx, double vy0, double dvy, int nvy, int mode, int32_t* sx,
                        int32_t* sy, float* fx, float* fy, cudaStream_t s);

// Sky statistics (FP64, deterministic) and normalisation/conversion.
//   partial: workspace of sky_partial_doubles(N) doubles.
size_t sky_partial_doubles(int N);
int launch_normalize(const float* raw, int N, int64_t npix, int normalize, float cr_clip,
                     int storage, void* cube, double* mu, double* sigma, double* partial,
                     cudaStream_t s);

// Generic stack kernels over velocity indices [k0, k0+nk): threshold ->
// pending list; optional dump of S and n_cov for the listed velocities.
int launch_stack_generic(const FieldDev& fd, int mode, int k0, int nk, const int32_t* dump_k,
                         float* dump_S, int32_t* dump_C, Pending* pend, int64_t pend_cap,
                         Counters* ctr, cudaStream_t s);

// Register-window stack kernel (nearest or bilinear sampling); returns -1 when
// the field's geometry does not fit the kernel (caller falls back).
struct FastPlan;
int fast_plan_size_bytes();
int fast_num_variants();
int fast_num_variants_for(const FastPlan* fp, int storage);
int fast_get_variant(const FastPlan* fp);
int fast_autotune(const FieldDev& fd, FastPlan* fp, int64_t items, Pending* pend,
                  int64_t pend_cap, Counters* ctr, cudaStream_t s);
const char* fast_variant_name(const FastPlan* fp, int storage);
void fast_set_variant(FastPlan* fp, int v);
// Whether the field can use the fast kernel at all (width a multiple of
// 16 bytes for the tensor map).
bool fast_eligible(const FieldDev& fd, int mode);
// Builds the per-frame tile tables for the current shift tables; *fits tells
// whether the motion spans fit the kernel.  Synchronises the stream.
int fast_prepare(const FieldDev& fd, FastPlan* fp, cudaStream_t s, bool* fits);
bool fast_plan_build(const FieldDev& fd, int mode, FastPlan** out);
void fast_plan_free(FastPlan* fp);
int launch_stack_fast(const FieldDev& fd, const FastPlan* fp, int k0, int nk,
                      const int32_t* dump_k, float* dump_S, int32_t* dump_C, Pending* pend,
                      int64_t pend_cap, Counters* ctr, cudaStream_t s);
// One persistent launch over n prepared, fitting fields (same storage and
// sampling; the variant of fps[0]), items taken longest field first.
// Encodes and uploads the tensor maps a launch over these fields needs (so the
// launch itself copies nothing); *restaged tells whether any map changed.
bool fast_stage(const FieldDev* fds, FastPlan* const* fps, int n, cudaStream_t s,
                bool* restaged);
int launch_stack_fast_multi(const FieldDev* fds, FastPlan* const* fps, int n, float* dump_S,
                            int32_t* dump_C, Pending* pend, int64_t pend_cap, Counters* ctr,
                            cudaStream_t s);

// Local-maximum test of the pending points -> candidate list (unsorted) and keys.
int launch_resolve(const FieldDev* fds_dev, int n_fields, int mode, const Pending* pend,
                   const Counters* ctr, int64_t pend_cap, st_candidate* cand,
                   uint64_t* keys, uint32_t* idx, int64_t cand_cap, Counters* ctr_out,
                   cudaStream_t s);

// Sorts keys/idx (n_pow2 entries, padded with ~0) and gathers the first
// `capacity` records into out.
int launch_sort_gather(uint64_t* keys, uint32_t* idx, int64_t n_pow2, const Counters* ctr,
                       const st_candidate* cand, st_candidate* out, int64_t capacity,
                       cudaStream_t s);
int launch_pad_keys(uint64_t* keys, uint32_t* idx, int64_t n_pow2, const Counters* ctr,
                    cudaStream_t s);

// Refinement: optimise == false evaluates J, SNR and (optionally) dJ/dtheta at
// the given theta; optimise == true runs `steps` Adam steps from each
// candidate's grid velocity and pixel, with F at its optimum, and writes the
// refined records.
// Refinement (forward + adjoint, optional Adam steps) of n candidates; h_fds
// are the host copies of the n_fields device descriptors fds (their cubes are
// mapped for TMA into d_maps, n_fields entries).  Returns -1 if a field cannot
// be mapped or has more than refine_max_frames() frames.
int refine_max_frames();
int launch_refine(const FieldDev* h_fds, int n_fields, const FieldDev* fds, CUtensorMap* d_maps,
                  const double* const* times, const double* t_ref, const double* grid,
                  int storage, bool optimise, const float* theta, const int32_t* centre,
                  const int32_t* field, const st_candidate* cand, int64_t n, int steps,
                  int optimizer, float fwhm, float lr_pos, float lr_vel, float* J, float* snr,
                  float* grad, st_refined* out, int* err, cudaStream_t s);

// Tracks: links the sorted candidates [n] into components (workspace of
// link_workspace_bytes(n) bytes); writes up to cap tracks, *n_tracks = all.
// Synchronises s.  Returns launches or -1.
int64_t link_workspace_bytes(int64_t n);
int launch_link_tracks(const st_candidate* c, int64_t n, const FieldDev* fds, const double* grid,
                       int r_xy, int r_v, void* ws, st_track* out, int64_t cap,
                       int64_t* n_tracks, cudaStream_t s);

// Front end (Sec. 2.1): median star removal over a group of N frames (N <=
// median_max_frames()), sums of every n_sum frames into M outputs, 2 x 2
// binning.  Each returns the number of launches or -1 if the sizes exceed
// the launch limits.
int median_max_frames();
int median_select_max_frames();
int launch_median_select(const float* in, int N, int64_t P, float* out, float* median,
                         cudaStream_t s);
int launch_median_subtract(const float* in, int N, int64_t P, float* out, float* median,
                           cudaStream_t s);
int launch_sum_frames(const float* in, int n_sum, int M, int64_t P, float* out, cudaStream_t s);
int launch_bin2x2(const float* in, int N, int H, int W, float* out, cudaStream_t s);

// Tiled TMA map of a field's cube [N][H][W] (storage type) with a box of
// box_w x box_h x 1 elements, zero fill outside.  False if it cannot be built.
bool encode_tile_map(CUtensorMap* map, const FieldDev& fd, int box_w, int box_h);

}  // namespace st
