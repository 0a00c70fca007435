/*
 * st.h — C ABI of the GB300 synthetic-tracking (shift-and-stack) library.
 *
 * Method (Burdanov, Hasler & de Wit 2023, "GPU-based framework for detecting
 * small Solar System bodies in targeted exoplanet surveys"):
 *   Sec. 1   shift-and-stack: remove stationary sources, predict a linear
 *            motion, shift each image along it and combine the shifted images;
 *            synthetic tracking repeats this over a blind grid of motions.
 *   Sec. 2.1 (Last-night data) the frames are shifted and summed with no
 *            constraint on position angle, assuming linear motion; the
 *            slowest motion is set by the minimum shift (about 0.5 px); the
 *            output is a set of tracks with speed, position angle, pixel
 *            coordinates and S/N; an object must stand above the threshold
 *            in at least half of the images.
 *
 * Everything below runs on one CUDA device.  All pointers named d_* are
 * device pointers and h_* are host pointers.  The caller owns every buffer it
 * passes in; the plan owns its own workspace.  No call throws: each returns an
 * st_status, and st_last_error() gives a message for the calling thread.
 *
 * Definitions shared by every entry point (the library's reading of Sec. 2.1):
 *   dt_i      = t_i - t_ref, in FP64.
 *   v(a,b)    = (vx0 + a*dvx, vy0 + b*dvy), a in [0,nvx), b in [0,nvy);
 *               linear velocity index k = b*nvx + a.
 *   nearest   : sx(i,a) = floor(vx_a*dt_i + 0.5), sy(i,b) likewise, FP64,
 *               no fused multiply-add.
 *   stack     : S_k(x,y) = sum_{i=0..N-1} I_i(x+sx(i,a), y+sy(i,b)), the sum
 *               taken in FP32 in frame order i = 0..N-1 with one accumulator;
 *               samples outside the frame contribute +0.0.
 *   coverage  : n_cov(x,y,k) = number of frames whose sample is inside.
 *   bilinear  : the shift s = v*dt_i is split into floor(s) and a fraction f;
 *               the sample interpolates the four taps around x+floor(s) with
 *               weights (1-fx, fx) x (1-fy, fy); taps outside read 0; the
 *               sample is inside iff 0 <= x+s <= W-1 and 0 <= y+s_y <= H-1.
 *   candidate : n_cov >= n_min (n_min = ceil(N/2) unless given), and
 *               S >= thr[n_cov] with thr[n] = (float)(tau*sqrt((double)n)),
 *               and S is a local maximum of S_k over its 8 neighbours inside
 *               the frame whose n_cov >= n_min: strictly greater than the
 *               neighbours that come earlier in raster order (y, then x) and
 *               greater or equal to the later ones.
 *   snr       : S * (float)(1/sqrt((double)n_cov)), in FP32.
 *   order     : candidates are returned sorted by (field, k, y, x).
 */
#ifndef ST_H_
#define ST_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ST_VERSION_MAJOR 0
#define ST_VERSION_MINOR 1

typedef enum {
  ST_OK = 0,
  ST_ERR_INVALID = 1,     /* an argument is out of range; nothing was launched */
  ST_ERR_CUDA = 2,        /* a CUDA runtime call failed; message has the CUDA error */
  ST_ERR_OOM = 3,         /* device or pinned-host allocation failed; nothing leaked */
  ST_ERR_OVERFLOW = 4,    /* more candidates than capacity; *h_count holds the true count */
  ST_ERR_TIMEOUT = 5,     /* a bounded device wait ran out; the device stays usable */
  ST_ERR_UNSUPPORTED = 6  /* valid request this build does not implement */
} st_status;

typedef enum { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 } st_dtype;
typedef enum { ST_NEAREST = 0, ST_BILINEAR = 1 } st_shift;

/* One field: a cube of n_frames frames of width x height pixels, row-major
 * [n_frames][height][width], and the velocity grid searched over it.
 * Velocities are in pixels per unit of the timestamps. */
typedef struct {
  int32_t width, height, n_frames;
  double t_ref;              /* reference epoch; same unit as the timestamps */
  double vx0, dvx;           /* x velocity grid: vx_a = vx0 + a*dvx */
  int32_t nvx;
  double vy0, dvy;           /* y velocity grid: vy_b = vy0 + b*dvy */
  int32_t nvy;
  float snr_threshold;       /* tau, in units of the per-frame noise sigma */
  int32_t min_coverage;      /* n_min; 0 selects ceil(n_frames/2) (Sec. 2.1) */
} st_field;

typedef struct {
  st_dtype storage;          /* frame storage type on the device; sums are always FP32 */
  st_shift mode;             /* ST_NEAREST or ST_BILINEAR */
  int32_t normalize;         /* 1: per-frame robust sky mean/sigma in FP64 and
                                I = (R - mu)/sigma, NaN -> 0; 0: frames are used
                                as given (NaN propagates) */
  float cr_clip;             /* with normalize: zero |I| > cr_clip; 0 disables */
  int32_t use_graph;         /* 1: the device part of a search (normalisation,
                                the stack launch, local maxima, counters) is
                                captured into a CUDA graph on the first call
                                with given frame pointers and timestamps and
                                replayed while both stay the same (shift tables
                                are rebuilt only when the timestamps change) */
  int32_t tile;              /* stack kernel: -1 = register-window variant chosen
                                by timing the variants on the field with the most
                                work (cached in tune_cache), 0 = default variant,
                                1 = direct-gather kernel only, 2.. = register-
                                window variant (tile - 2) of the list for the
                                storage type and sampling (out of range: 0); a
                                field whose motion does not fit the window takes
                                the direct-gather kernel */
  const char* tune_cache;    /* JSON file for autotuned tiles, or NULL */
  int64_t pending_capacity;  /* above-threshold points held before the local-max
                                test; 0 selects a default of 4 Mi points */
} st_opts;

/* One detection (Sec. 2.1: pixel coordinates, velocity and S/N). 28 bytes. */
typedef struct {
  int32_t x, y;              /* pixel in reference-epoch coordinates */
  int32_t k;                 /* velocity index, k = b*nvx + a */
  int32_t field;             /* index of the field in the plan */
  float stack;               /* S_k(x, y) */
  float snr;                 /* S * (1/sqrt(n_cov)) */
  int32_t n_cov;             /* frames covering the pixel */
} st_candidate;

/* One track: the linked detections of one object (Sec. 2.1 returns tracks
 * with speed, PA, pixel coordinates and S/N), represented by its detection
 * of highest S/N.  48 bytes. */
typedef struct {
  int32_t x, y;              /* pixel of the representative detection */
  int32_t k;                 /* its velocity index */
  int32_t field;
  float stack, snr;          /* its stack value and S/N */
  int32_t n_cov;             /* its coverage */
  int32_t members;           /* detections linked into the track */
  float vx, vy;              /* grid velocity of the representative, px per time unit */
  float speed;               /* hypot(vx, vy) */
  float pa;                  /* degrees in [0, 360), from -y towards -x (north up, east left) */
} st_track;

/* One refined detection: continuous motion and position at t_ref. */
typedef struct {
  float vx, vy, x0, y0, flux;
  float snr;                 /* matched-filter S/N at the final parameters */
  float obj;                 /* objective J at the final parameters */
  int32_t field;
} st_refined;

typedef struct st_plan_s st_plan_t;

/* Library version as MAJOR*100 + MINOR. */
int32_t st_version(void);

/* Message of the last failing call on this thread; valid until the next call
 * on the same thread.  Never NULL. */
const char* st_last_error(void);

/* Builds a plan for n_fields fields: validates them, sizes the workspace,
 * allocates it on the current device and picks the stack tile variant.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream) on which every
 * later call on this plan is ordered.  Limits: width, height <= 16384,
 * n_frames <= 65535 (one grid row per frame in the normalisation kernels),
 * nvx*nvy <= 2^26, n_fields <= 255.  On failure *out is NULL and nothing is
 * left allocated. */
st_status st_plan(const st_field* fields, int32_t n_fields, const st_opts* opts,
                  void* cuda_stream, st_plan_t** out);

/* Releases the plan and its workspace.  NULL-safe. Synchronises the plan's stream. */
void st_free(st_plan_t* plan);

/* The search of Sec. 2.1 over every field of the plan: shift tables, optional
 * normalisation, shift-and-stack over the whole grid, threshold, local maxima,
 * and the sorted candidate list.
 *   d_frames[f]: device FP32 cube of field f, [N][H][W] row-major, read-only.
 *   h_times[f] : host FP64 timestamps of field f, [N].
 *   d_out      : device array of `capacity` candidates (may be NULL if capacity 0).
 *   h_count    : receives the total number of candidates found.
 * Synchronises the plan's stream (to read the count).  Returns ST_ERR_OVERFLOW
 * when the total exceeds capacity: the first `capacity` records of the sorted
 * list are written and *h_count holds the total, so a retry with a larger
 * buffer succeeds.  Returns ST_ERR_OVERFLOW with *h_count = -1 when the
 * above-threshold points exceed the plan's pending_capacity, and
 * ST_ERR_TIMEOUT (*h_count = -1) when a pipeline wait of the stack kernel
 * gave up after 2 s (the device stays usable).  Every field whose motion fits
 * the register-window kernel is searched in one persistent launch; shift
 * tables are rebuilt only when a field's timestamps change. */
st_status st_stack_search(st_plan_t* plan, const float* const* d_frames,
                          const double* const* h_times, st_candidate* d_out,
                          int64_t capacity, int64_t* h_count);

/* Same search with host buffers: h_frames[f] are host FP32 cubes (pinned or
 * pageable) copied to the device inside the call, and the sorted candidates
 * are copied back into h_out (capacity records).  The plan holds the device
 * copies, allocated on the first call. */
st_status st_stack_search_host(st_plan_t* plan, const float* const* h_frames,
                               const double* const* h_times, st_candidate* h_out,
                               int64_t capacity, int64_t* h_count);

/* Differentiable refinement of candidates (not in the paper; a continuous
 * refinement of grid detections).  For each input candidate of field f the
 * parameters theta = (vx, vy, x0, y0, F) start at the grid velocity, the pixel
 * and F = S/(N<g,g>); the objective on a 64x64 output cutout centred on the
 * starting pixel is
 *     J = F*<g, S_theta> - 0.5*F^2*N*<g, g>,
 * with S_theta the bilinear stack of the raw cube (FP32 input frames of the
 * plan's last search, normalised when the plan normalises) and g a Gaussian
 * of the given FWHM centred on (x0, y0).  `steps` optimiser steps maximise J,
 * each with F first set to its optimum <g,S>/(N<g,g>):
 *   optimizer 0 = Adam, learning rate lr_pos px for x0, y0 and lr_vel for
 *                 vx, vy;
 *   optimizer 1 = Gauss-Newton: (vx, vy, x0, y0) move by the solution of
 *                 (Hs + lr_pos * diag(Hs)) delta = dJ/d(vx, vy, x0, y0), Hs
 *                 the model's J^T J with F profiled out (Schur complement),
 *                 lr_pos >= 0 the damping; lr_vel is not used.
 * The frames' shifts v*(t_i - t_ref) are formed in FP64.
 * d_in: device candidates; d_out: device results [n]; d_grad_out: optional
 * device [n][5] gradient dJ/dtheta at the final parameters (order vx, vy, x0,
 * y0, F).  Requires a prior st_stack_search on the plan (frames resident).
 * The frames are staged per candidate by TMA tile copies: returns
 * ST_ERR_UNSUPPORTED when a field's row (width x element size) is not a
 * multiple of 16 bytes, it has more than 8192 frames or n exceeds 2^31 - 1
 * (one thread block per candidate), ST_ERR_INVALID for another optimizer or
 * a negative damping, and ST_ERR_TIMEOUT when a copy does not land within
 * 2 s (the kernel exits cleanly).  Synchronises the plan's stream. */
st_status st_refine(st_plan_t* plan, const st_candidate* d_in, int64_t n,
                    int32_t steps, int32_t optimizer, float fwhm, float lr_pos,
                    float lr_vel, st_refined* d_out, float* d_grad_out);

/* Forward and adjoint of the refinement objective for explicit parameters, the
 * building block of the autograd binding.  theta: device [n][5] (vx, vy, x0,
 * y0, F); centre: device [n][2] int32 cutout centres; fields: device [n]
 * int32.  Writes J [n], SNR [n] and, if d_grad is not NULL, dJ/dtheta [n][5].
 * Frames are those of the plan's last search; errors as st_refine. */
st_status st_refine_eval(st_plan_t* plan, const float* d_theta,
                         const int32_t* d_centre, const int32_t* d_field,
                         int64_t n, float fwhm, float* d_J, float* d_snr,
                         float* d_grad);

/* Search of one field that allocates no memory (the paper has no counterpart:
 * this serves callers that cannot allocate device memory when they search:
 * processes whose device memory is reserved up front by another allocator,
 * such as a framework's caching allocator that holds the free memory, and
 * hosts that forbid cudaMalloc after start-up because it can synchronise the
 * device and take unbounded time).  Same kernels, definitions and sorted output as st_stack_search
 * with normalize = 0 and FP32 storage, for one field (field index 0 in the
 * records).
 *   field      : the field (limits as st_plan: width, height <= 16384,
 *                n_frames <= 65535, nvx*nvy <= 2^26); mode: ST_NEAREST or
 *                ST_BILINEAR.
 *   d_frames   : device FP32 cube [N][H][W], used as given (not normalised).
 *   h_times    : host FP64 timestamps [N].
 *   d_out      : device array of `capacity` candidates (caller-owned).
 *   h_count    : receives the total number of candidates.
 *   cuda_stream: cudaStream_t on which the work is ordered; the call
 *                synchronises it to read the count.
 * Scratch: one 32 MiB device array inside the library, held by every GPU that
 * loads the library until the process exits.  It holds the shift tables
 * (16*N*(nvx+nvy) bytes plus small tables) and 64 bytes per above-threshold
 * slot; a field whose tables leave fewer than 1024 slots is rejected with
 * ST_ERR_INVALID, and more above-threshold points than slots gives
 * ST_ERR_OVERFLOW with *h_count = -1.  No call allocates: the first call on
 * each device (with that device current) looks up the array's device address
 * and caches it, so make that first call before any stream capture.  Every
 * call reuses the same array and the previous call's contents stay in it
 * (counters are cleared on each call); calls that overlap on the GPU, from
 * several streams or threads at once, race on it and must be serialised by
 * the caller. */
st_status st_stack_search_noalloc(const st_field* field, int32_t mode, const float* d_frames,
                                  const double* h_times, st_candidate* d_out, int64_t capacity,
                                  int64_t* h_count, void* cuda_stream);

/* Diagnostics used by the tests and the benchmark (not part of the search's
 * interface). */

/* Shift tables of field f for timestamps h_times: h_sx [N][nvx], h_sy [N][nvy]
 * (nearest mode: the rounded shifts; bilinear: floor of the shift) and, if
 * not NULL, h_fx [N][nvx], h_fy [N][nvy] the FP32 fractions.  Computed by the
 * device kernel of the search. */
st_status st_shift_tables(st_plan_t* plan, int32_t field, const double* h_times,
                          int32_t* h_sx, int32_t* h_sy, float* h_fx, float* h_fy);

/* Robust sky statistics and normalisation alone (field f):  d_frames as in
 * st_stack_search; writes the storage cube into d_cube (device, N*H*W elements
 * of the plan's storage type) and per-frame h_mu, h_sigma (host, [N]). */
st_status st_normalize(st_plan_t* plan, int32_t field, const float* d_frames,
                       void* d_cube, double* h_mu, double* h_sigma);

/* Full stack planes S_k and n_cov for the n_k velocity indices h_k of field f,
 * computed by the search kernel: d_S [n_k][H][W] FP32, d_ncov [n_k][H][W]
 * int32 (may be NULL).  Frames are processed exactly as by st_stack_search. */
st_status st_dump_stack(st_plan_t* plan, int32_t field, const float* d_frames,
                        const double* h_times, const int32_t* h_k, int32_t n_k,
                        float* d_S, int32_t* d_ncov);

/* Number of the library's own kernel launches issued by the last
 * st_stack_search / st_stack_search_host / st_refine call on this plan. */
int64_t st_last_launch_count(const st_plan_t* plan);

/* Average device time in milliseconds of the main stack kernel over the last
 * search call (CUDA events on the plan's stream), and its launch count. */
st_status st_last_stack_kernel_time(const st_plan_t* plan, double* ms, int64_t* launches);

/* Which stack kernel field f used in the last search on this plan:
 * 1 = register-window kernel, 0 = direct-gather kernel, -1 = no search yet. */
int32_t st_last_stack_variant(const st_plan_t* plan, int32_t field);

/* Name of the stack kernel field f used in the last search on this plan:
 * "direct-gather", the register-window variant's name (storage type, rows
 * per thread, ring stages, frames per stage, column pairs, code options:
 * o16 the generated item loop, o48 the same with two x-velocities a thread;
 * x-velocity tiles per block), or "?" before any search.  The string is
 * static (owned by the library). */
const char* st_stack_variant_name(const st_plan_t* plan, int32_t field);

/* 1 if the device part of the last search (normalisation, stack, local
 * maxima) ran as a CUDA graph (use_graph: captured on the first search with
 * given frame pointers and timestamps, replayed while they stay the same),
 * 0 otherwise. */
int32_t st_last_graph_replayed(const st_plan_t* plan);

/* Links the detections of the plan's last search into tracks: two
 * detections of a field are linked when their pixels differ by at most r_xy
 * in x and y and their velocity indices by at most r_v in a and b; a track
 * is a connected component, reported with its detection of highest S/N
 * (ties: the first in (field, k, y, x) order) and its size, tracks in the
 * order of their first detection.  d_cand: device candidates [n] in the
 * order st_stack_search returns them; d_tracks: device [capacity]; *h_count
 * receives the number of tracks (ST_ERR_OVERFLOW if above capacity: the
 * first capacity tracks are written).  Synchronises the plan's stream. */
st_status st_link_tracks(st_plan_t* plan, const st_candidate* d_cand, int64_t n, int32_t r_xy,
                         int32_t r_v, st_track* d_tracks, int64_t capacity, int64_t* h_count);

/* ---- Pre-tracking front end (Sec. 2.1) --------------------------------
 * Device FP32 cubes [N][H][W] row-major, caller-owned; the calls are
 * asynchronous on cuda_stream (NULL: the legacy default stream) and allocate
 * nothing.  Errors: ST_ERR_INVALID for NULL pointers, sizes <= 0 or (sums,
 * binning) an output overlapping the input; ST_ERR_CUDA for a launch error. */

/* Median star removal: d_out[i] = d_in[i] - m for every frame i, with m the
 * per-pixel median over the N frames of the finite samples (NaN marks a
 * masked sample; an even count takes (a + b) * 0.5 of the two middle values;
 * a pixel with no finite sample gives NaN).  d_out may be d_in.  d_median
 * [H][W] (may be NULL) receives m.  N <= 768, else ST_ERR_UNSUPPORTED. */
st_status st_median_subtract(const float* d_in, int32_t n_frames, int32_t height,
                             int32_t width, float* d_out, float* d_median, void* cuda_stream);

/* Sums of every n_sum consecutive frames, in frame order with one FP32
 * accumulator: M = floor(N / n_sum) frames into d_out [M][H][W] (a trailing
 * partial group is dropped, so every sum has the same exposure).  h_times_out
 * [M] (host, may be NULL) receives the FP64 mean of each group's h_times
 * (h_times may be NULL when h_times_out is). */
st_status st_sum_frames(const float* d_in, int32_t n_frames, int32_t height, int32_t width,
                        int32_t n_sum, const double* h_times, float* d_out,
                        double* h_times_out, void* cuda_stream);

/* 2 x 2 binning: d_out [N][H/2][W/2] = ((p00 + p01) + p10) + p11 per block
 * (flux kept); an odd last row or column is dropped. */
st_status st_bin2x2(const float* d_in, int32_t n_frames, int32_t height, int32_t width,
                    float* d_out, void* cuda_stream);

/* FP32 add-rate microbenchmark (the roof of the nearest-shift stack): one
 * block of 1024 threads per SM, 16 independent add chains per thread, iters
 * iterations.  variant 0: scalar add.rn.f32; 1: paired add.rn.f32x2;
 * 2: paired adds interleaved 1:1 with integer adds.  Writes the median adds
 * per SM clock (from clock64) and the device-wide rate in T adds/s (CUDA
 * events).  Allocates and frees its own small buffers. */
st_status st_probe_add_rate(int32_t variant, int32_t iters, double* adds_per_clk_per_sm,
                            double* tadds_per_s);

/* Failure-detection probe: one thread waits, with the bounded wait every
 * pipeline of the library uses, on an mbarrier phase that nothing completes,
 * and gives up after limit_us microseconds (1 .. 2 000 000).  *h_timed_out
 * receives 1 when the wait ran out (the expected outcome), *h_waited_us the
 * time the kernel measured.  The context stays usable afterwards. */
st_status st_probe_wait_timeout(int32_t limit_us, int32_t* h_timed_out, double* h_waited_us);

#ifdef __cplusplus
}
#endif

#endif /* ST_H_ */
