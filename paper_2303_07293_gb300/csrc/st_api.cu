// st_api.cu — the C ABI of include/st.h: plan, search, diagnostics.
//
// The search of Sec. 2.1 (Burdanov, Hasler & de Wit 2023) runs as:
//   shift tables (FP64 dt_i = t_i - t_ref)  ->  optional robust normalisation
//   ->  shift-and-stack + threshold (stack kernels)  ->  local maxima
//   ->  sort by (field, k, y, x)  ->  caller's buffer.
// Every step is a kernel of this library; the host only validates, sizes
// workspace, launches and reads the candidate count.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "st_internal.h"

using namespace st;

namespace {

thread_local std::string g_err = "no error";

st_status fail(st_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      if (e_ == cudaErrorMemoryAllocation)                                            \
        return fail(ST_ERR_OOM, "%s: %s", #call, cudaGetErrorString(e_));             \
      return fail(ST_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));              \
    }                                                                                 \
  } while (0)

int64_t pow2_at_least(int64_t n) {
  int64_t p = 1;
  while (p < n) p <<= 1;
  return p;
}

}  // namespace

namespace st {
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace st

struct FieldPlan {
  st_field f{};
  int nmin = 0;
  double* d_t = nullptr;
  int32_t* d_sx = nullptr;
  int32_t* d_sy = nullptr;
  float* d_fx = nullptr;
  float* d_fy = nullptr;
  float* d_thr = nullptr;
  float* d_rsq = nullptr;
  void* d_cube = nullptr;        // normalised / converted storage cube (owned)
  float* d_frames_copy = nullptr; // device copy for the host-buffer entry point
  FastPlan* fast = nullptr;
  int last_variant = -1;
  bool tuned = false;
  const float* last_frames = nullptr;
  std::vector<double> h_t;     // timestamps the shift tables were built for
  bool tables_valid = false;   // shift tables match h_t
  bool fast_ready = false;     // register-window tables built for the current shift tables
  bool fast_fits = false;      // and the field's motion fits the kernel
  int64_t P() const { return (int64_t)f.width * f.height; }
  int64_t nk() const { return (int64_t)f.nvx * f.nvy; }
};

struct st_plan_s {
  std::vector<FieldPlan> F;
  st_opts o{};
  cudaStream_t s = nullptr;
  int device = 0;
  Pending* d_pend = nullptr;
  int64_t pend_cap = 0;
  Counters* d_ctr = nullptr;
  Counters* h_ctr = nullptr;  // pinned
  st_candidate* d_cand = nullptr;
  uint64_t* d_keys = nullptr;
  uint32_t* d_idx = nullptr;
  int64_t sort_cap = 0;
  FieldDev* d_fds = nullptr;
  double** d_times = nullptr;  // per field: device pointer to its timestamps
  double* d_tref = nullptr;    // per field
  double* d_grid = nullptr;    // per field: vx0, dvx, vy0, dvy
  CUtensorMap* d_maps = nullptr;  // per field: TMA map of the cube for the refinement
  void* d_link_ws = nullptr;      // track-linking workspace
  int64_t link_ws_bytes = 0;
  int* d_rerr = nullptr;          // refinement timeout flag
  double* d_sky = nullptr;
  st_candidate* d_hout = nullptr;
  int64_t hout_cap = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  std::string tune_cache;
  int sms = 0;
  double stack_ms = 0.0;
  int64_t stack_launches = 0;
  int64_t launches = 0;
  bool has_search = false;
  // CUDA graph of the device part of a search (normalise, stack, resolve),
  // valid for the frame pointers and table generation it was captured with
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap_s = nullptr;  // capture stream (the plan's stream may be the legacy one)
  std::vector<const float*> graph_frames;
  uint64_t graph_gen = 0;
  uint64_t gen = 1;             // bumped when tables, variants or maps change
  int64_t graph_stack_launches = 0;
  int64_t graph_launches = 0;
  bool graph_broken = false;    // capture failed once: run directly
  bool last_replayed = false;
};

namespace {

void free_plan(st_plan_t* p) {
  if (!p) return;
  if (p->s) cudaStreamSynchronize(p->s);
  for (auto& fp : p->F) {
    cudaFree(fp.d_t);
    cudaFree(fp.d_sx);
    cudaFree(fp.d_sy);
    cudaFree(fp.d_fx);
    cudaFree(fp.d_fy);
    cudaFree(fp.d_thr);
    cudaFree(fp.d_rsq);
    cudaFree(fp.d_cube);
    cudaFree(fp.d_frames_copy);
    if (fp.fast) fast_plan_free(fp.fast);
  }
  if (p->graph) cudaGraphExecDestroy(p->graph);
  if (p->cap_s) cudaStreamDestroy(p->cap_s);
  cudaFree(p->d_pend);
  cudaFree(p->d_ctr);
  cudaFree(p->d_maps);
  cudaFree(p->d_rerr);
  cudaFree(p->d_link_ws);
  if (p->h_ctr) cudaFreeHost(p->h_ctr);
  cudaFree(p->d_cand);
  cudaFree(p->d_keys);
  cudaFree(p->d_idx);
  cudaFree(p->d_fds);
  cudaFree(p->d_times);
  cudaFree(p->d_tref);
  cudaFree(p->d_grid);
  cudaFree(p->d_sky);
  cudaFree(p->d_hout);
  if (p->e0) cudaEventDestroy(p->e0);
  if (p->e1) cudaEventDestroy(p->e1);
  delete p;
}

st_status validate_field(const st_field& f, int idx) {
  if (f.width <= 0 || f.height <= 0 || f.width > 16384 || f.height > 16384)
    return fail(ST_ERR_INVALID, "field %d: width/height must be in [1, 16384]", idx);
  if (f.n_frames <= 0 || f.n_frames > 65535)  // frames index grid rows (at most 65535)
    return fail(ST_ERR_INVALID, "field %d: n_frames must be in [1, 65535]", idx);
  if (f.nvx <= 0 || f.nvy <= 0 || (int64_t)f.nvx * f.nvy > (1ll << 26))
    return fail(ST_ERR_INVALID, "field %d: nvx, nvy >= 1 and nvx*nvy <= 2^26", idx);
  if (!std::isfinite(f.t_ref) || !std::isfinite(f.vx0) || !std::isfinite(f.dvx) ||
      !std::isfinite(f.vy0) || !std::isfinite(f.dvy))
    return fail(ST_ERR_INVALID, "field %d: grid and t_ref must be finite", idx);
  if (!std::isfinite(f.snr_threshold) || f.snr_threshold < 0.0f)
    return fail(ST_ERR_INVALID, "field %d: snr_threshold must be finite and >= 0", idx);
  if (f.min_coverage < 0 || f.min_coverage > f.n_frames)
    return fail(ST_ERR_INVALID, "field %d: min_coverage must be in [0, n_frames]", idx);
  return ST_OK;
}

st_status check_times(const double* t, int N, const st_field& f, int idx) {
  if (!t) return fail(ST_ERR_INVALID, "field %d: timestamps are NULL", idx);
  for (int i = 0; i < N; ++i)
    if (!std::isfinite(t[i])) return fail(ST_ERR_INVALID, "field %d: timestamp %d not finite", idx, i);
  // |v * dt| must stay inside int32 shifts
  double vmax = std::max(std::max(std::fabs(f.vx0), std::fabs(f.vx0 + (f.nvx - 1) * f.dvx)),
                         std::max(std::fabs(f.vy0), std::fabs(f.vy0 + (f.nvy - 1) * f.dvy)));
  for (int i = 0; i < N; ++i)
    if (vmax * std::fabs(t[i] - f.t_ref) > 1e9)
      return fail(ST_ERR_INVALID, "field %d: shift of frame %d exceeds 1e9 px", idx, i);
  return ST_OK;
}

size_t store_bytes(int storage) { return storage == ST_F32 ? 4 : 2; }

// Autotuning cache: a flat JSON object {"<field key>": variant, ...}.
std::string tune_key(const st_field& f, int storage, int mode, int sms) {
  char b[160];
  snprintf(b, sizeof b, "W%d_H%d_N%d_nvx%d_nvy%d_st%d_m%d_sm%d", f.width, f.height, f.n_frames,
           f.nvx, f.nvy, storage, mode, sms);
  return b;
}

int tune_lookup(const std::string& path, const std::string& key) {
  if (path.empty()) return -1;
  FILE* fh = fopen(path.c_str(), "r");
  if (!fh) return -1;
  std::string txt;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, fh)) > 0) txt.append(buf, n);
  fclose(fh);
  size_t at = txt.find("\"" + key + "\"");
  if (at == std::string::npos) return -1;
  at = txt.find(':', at);
  if (at == std::string::npos) return -1;
  return atoi(txt.c_str() + at + 1);
}

void tune_store(const std::string& path, const std::string& key, int variant) {
  if (path.empty()) return;
  std::string txt;
  if (FILE* fh = fopen(path.c_str(), "r")) {
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, fh)) > 0) txt.append(buf, n);
    fclose(fh);
  }
  char entry[256];
  snprintf(entry, sizeof entry, "\"%s\": %d", key.c_str(), variant);
  const size_t at = txt.find("\"" + key + "\"");
  const size_t close = txt.rfind('}');
  if (at != std::string::npos) {
    // the key is there with a value this build cannot use: replace the value
    const size_t end = txt.find_first_of(",}", at);
    if (end == std::string::npos) return;
    txt = txt.substr(0, at) + entry + txt.substr(end);
  } else if (close == std::string::npos || txt.find('"') == std::string::npos) {
    txt = std::string("{") + entry + "}\n";
  } else {
    txt = txt.substr(0, close) + ", " + entry + "}\n";
  }
  if (FILE* fh = fopen(path.c_str(), "w")) {
    fputs(txt.c_str(), fh);
    fclose(fh);
  }
}

// Shift tables of field fi for the given timestamps; rebuilt only when the
// timestamps differ from those of the current tables.
st_status prepare_tables(st_plan_t* p, int fi, const double* h_times, int64_t* launches,
                         bool* changed) {
  FieldPlan& fp = p->F[fi];
  const st_field& f = fp.f;
  st_status st = check_times(h_times, f.n_frames, f, fi);
  if (st != ST_OK) return st;
  *changed = false;
  if (fp.tables_valid && fp.h_t.size() == (size_t)f.n_frames &&
      std::memcmp(fp.h_t.data(), h_times, sizeof(double) * f.n_frames) == 0)
    return ST_OK;
  CK(cudaMemcpyAsync(fp.d_t, h_times, sizeof(double) * f.n_frames, cudaMemcpyHostToDevice, p->s));
  *launches += launch_shift_tables(fp.d_t, f.n_frames, f.t_ref, f.vx0, f.dvx, f.nvx, f.vy0, f.dvy,
                                   f.nvy, p->o.mode, fp.d_sx, fp.d_sy, fp.d_fx, fp.d_fy, p->s);
  CK(cudaGetLastError());
  fp.h_t.assign(h_times, h_times + f.n_frames);
  fp.tables_valid = true;
  fp.fast_ready = false;
  ++p->gen;
  *changed = true;
  return ST_OK;
}

// Optional normalisation / storage conversion of field fi into the plan's cube.
int64_t normalize_field(st_plan_t* p, int fi, const float* d_frames) {
  FieldPlan& fp = p->F[fi];
  fp.last_frames = d_frames;
  if (!fp.d_cube) return 0;
  return launch_normalize(d_frames, fp.f.n_frames, fp.P(), p->o.normalize, p->o.cr_clip,
                          p->o.storage, fp.d_cube, nullptr, nullptr, p->d_sky, p->s);
}

// Tables + optional normalisation for field fi with the given frames/times.
st_status prepare_field(st_plan_t* p, int fi, const float* d_frames, const double* h_times,
                        int64_t* launches) {
  bool changed = false;
  st_status st = prepare_tables(p, fi, h_times, launches, &changed);
  if (st != ST_OK) return st;
  *launches += normalize_field(p, fi, d_frames);
  CK(cudaGetLastError());
  return ST_OK;
}

FieldDev field_dev(const FieldPlan& fp, const float* d_frames, int fi, int storage) {
  FieldDev d{};
  d.cube = fp.d_cube ? fp.d_cube : (const void*)d_frames;
  d.storage = fp.d_cube ? storage : ST_F32;
  d.W = fp.f.width;
  d.H = fp.f.height;
  d.N = fp.f.n_frames;
  d.nvx = fp.f.nvx;
  d.nvy = fp.f.nvy;
  d.nmin = fp.nmin;
  d.field = fi;
  d.sx = fp.d_sx;
  d.sy = fp.d_sy;
  d.fx = fp.d_fx;
  d.fy = fp.d_fy;
  d.thr = fp.d_thr;
  d.rsq = fp.d_rsq;
  return d;
}

st_status device_search(st_plan_t* p, const float* const* d_frames, const double* const* h_times,
                        st_candidate* d_out, int64_t capacity, int64_t* h_count) {
  if (!d_frames || !h_times || !h_count) return fail(ST_ERR_INVALID, "NULL argument");
  if (capacity < 0 || (capacity > 0 && !d_out))
    return fail(ST_ERR_INVALID, "capacity must be >= 0 and d_out non-NULL when capacity > 0");
  int nf = (int)p->F.size();
  for (int fi = 0; fi < nf; ++fi)
    if (!d_frames[fi]) return fail(ST_ERR_INVALID, "field %d: frames are NULL", fi);
  // ---- host-side preparation: tables (when the timestamps change), the
  // register-window tables and variant, the tensor maps
  int64_t L = 0;
  std::vector<FieldDev> fds(nf);
  for (int fi = 0; fi < nf; ++fi) {
    bool changed = false;
    st_status st = prepare_tables(p, fi, h_times[fi], &L, &changed);
    if (st != ST_OK) return st;
    fds[fi] = field_dev(p->F[fi], d_frames[fi], fi, p->o.storage);
  }
  CK(cudaMemcpyAsync(p->d_fds, fds.data(), sizeof(FieldDev) * nf, cudaMemcpyHostToDevice, p->s));
  // fields that fit the register-window kernel run in one persistent launch;
  // its variant is tuned (or looked up) on the field with the most work
  std::vector<char> use_fast(nf, 0);
  std::vector<FieldDev> fast_fds;
  std::vector<FastPlan*> fast_fps;
  int tune_fi = -1;
  for (int fi = 0; fi < nf; ++fi) {
    FieldPlan& fp = p->F[fi];
    if (fp.fast && !fp.fast_ready) {
      bool fits = false;
      L += fast_prepare(fds[fi], fp.fast, p->s, &fits);
      CK(cudaGetLastError());
      fp.fast_fits = fits;
      fp.fast_ready = true;
    }
    use_fast[fi] = fp.fast && fp.fast_fits;
    if (use_fast[fi]) {
      fast_fds.push_back(fds[fi]);
      fast_fps.push_back(fp.fast);
      const double work = (double)fp.P() * fp.f.n_frames * fp.nk();
      if (tune_fi < 0 || work > (double)p->F[tune_fi].P() * p->F[tune_fi].f.n_frames *
                                    p->F[tune_fi].nk())
        tune_fi = fi;
    }
  }
  if (tune_fi >= 0 && p->o.tile == -1) {
    FieldPlan& tp = p->F[tune_fi];
    if (!tp.tuned) {
      const std::string key = tune_key(tp.f, fds[tune_fi].storage, p->o.mode, p->sms);
      int v = tune_lookup(p->tune_cache, key);
      if (v >= 0 && v < fast_num_variants_for(tp.fast, fds[tune_fi].storage)) {
        fast_set_variant(tp.fast, v);
      } else {
        // the variants are timed on the field's frames as the search reads them
        L += normalize_field(p, tune_fi, d_frames[tune_fi]);
        L += fast_autotune(fds[tune_fi], tp.fast, 64ll * p->sms, p->d_pend, p->pend_cap,
                           p->d_ctr, p->s);
        tune_store(p->tune_cache, key, fast_get_variant(tp.fast));
      }
      tp.tuned = true;
      ++p->gen;
    }
    for (FastPlan* f : fast_fps) fast_set_variant(f, fast_get_variant(tp.fast));
  }
  if (!fast_fds.empty()) {
    // the field with the most work first: its variant is the launch's
    for (size_t i = 0; i < fast_fds.size(); ++i)
      if (fast_fds[i].field == tune_fi) {
        std::swap(fast_fds[0], fast_fds[i]);
        std::swap(fast_fps[0], fast_fps[i]);
      }
    bool restaged = false;
    if (!fast_stage(fast_fds.data(), fast_fps.data(), (int)fast_fds.size(), p->s, &restaged)) {
      for (int fi = 0; fi < nf; ++fi) use_fast[fi] = 0;  // every field: direct gather
      fast_fds.clear();
    }
    if (restaged) ++p->gen;
  }
  for (int fi = 0; fi < nf; ++fi) p->F[fi].last_variant = use_fast[fi] ? 1 : 0;

  // ---- the device part of the search: normalise, stack, resolve, counters.
  // Errors are collected, not returned, so that a capture always ends.
  bool capturing = false;
  auto record = [&](cudaEvent_t ev) {
    // inside a capture the timing events become event-record nodes of the graph
    return capturing ? cudaEventRecordWithFlags(ev, p->s, cudaEventRecordExternal)
                     : cudaEventRecord(ev, p->s);
  };
  auto issue = [&](int64_t* stack_launches, int64_t* launches) -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(p->d_ctr, 0, sizeof(Counters), p->s);
    for (int fi = 0; fi < nf; ++fi) *launches += normalize_field(p, fi, d_frames[fi]);
    if (e == cudaSuccess) e = record(p->e0);
    if (!fast_fds.empty()) {
      int n = launch_stack_fast_multi(fast_fds.data(), fast_fps.data(), (int)fast_fds.size(),
                                      nullptr, nullptr, p->d_pend, p->pend_cap, p->d_ctr, p->s);
      if (n < 0 && e == cudaSuccess) e = cudaErrorLaunchFailure;
      *stack_launches += n > 0 ? n : 0;
    }
    for (int fi = 0; fi < nf; ++fi)
      if (!use_fast[fi])
        *stack_launches += launch_stack_generic(fds[fi], p->o.mode, 0, (int)p->F[fi].nk(),
                                                nullptr, nullptr, nullptr, p->d_pend,
                                                p->pend_cap, p->d_ctr, p->s);
    if (e == cudaSuccess) e = record(p->e1);
    *launches += launch_resolve(p->d_fds, nf, p->o.mode, p->d_pend, p->d_ctr, p->pend_cap,
                                p->d_cand, p->d_keys, p->d_idx, p->pend_cap, p->d_ctr, p->s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->h_ctr, p->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, p->s);
    return e;
  };
  int64_t stack_launches = 0, dev_launches = 0;
  p->last_replayed = false;
  bool done = false;
  if (p->o.use_graph && !p->graph_broken) {
    std::vector<const float*> key(d_frames, d_frames + nf);
    if (!(p->graph && p->graph_gen == p->gen && p->graph_frames == key)) {
      // capture the device part once for these frames and tables
      if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
      }
      // captured on a plan-owned stream (the plan's own stream may be the
      // legacy default stream, which cannot be captured), launched on the
      // plan's stream
      cudaGraph_t g = nullptr;
      int64_t sl = 0, dl = 0;
      cudaError_t e = cudaSuccess;
      if (!p->cap_s) e = cudaStreamCreateWithFlags(&p->cap_s, cudaStreamNonBlocking);
      const cudaStream_t user_s = p->s;
      if (e == cudaSuccess) e = cudaStreamBeginCapture(p->cap_s, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        p->s = p->cap_s;
        capturing = true;
        cudaError_t e2 = issue(&sl, &dl);
        capturing = false;
        p->s = user_s;
        e = cudaStreamEndCapture(p->cap_s, &g);
        if (e == cudaSuccess) e = e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&p->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        set_last_error((std::string("graph capture failed, running directly: ") +
                        cudaGetErrorString(e)).c_str());
        cudaGetLastError();  // clear a capture error; run directly from now on
        if (p->graph) cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
        p->graph_broken = true;
      } else {
        p->graph_frames = key;
        p->graph_gen = p->gen;
        p->graph_stack_launches = sl;
        p->graph_launches = dl;
      }
    }
    if (p->graph) {
      CK(cudaGraphLaunch(p->graph, p->s));
      stack_launches = p->graph_stack_launches;
      dev_launches = p->graph_launches;
      p->last_replayed = true;
      done = true;
    }
  }
  if (!done) {
    cudaError_t e = issue(&stack_launches, &dev_launches);
    if (e != cudaSuccess) return fail(ST_ERR_CUDA, "search: %s", cudaGetErrorString(e));
  }
  L += stack_launches + dev_launches;
  CK(cudaStreamSynchronize(p->s));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, p->e0, p->e1));
  p->stack_ms = ms;
  p->stack_launches = stack_launches;
  Counters c = *p->h_ctr;
  if (c.error & ERR_PENDING_OVERFLOW) {
    *h_count = -1;
    p->launches = L;
    return fail(ST_ERR_OVERFLOW,
                "%llu above-threshold points exceed pending_capacity %lld; raise it in st_opts",
                (unsigned long long)c.n_pending, (long long)p->pend_cap);
  }
  if (c.error & ERR_TIMEOUT) {
    *h_count = -1;
    p->launches = L;
    return fail(ST_ERR_TIMEOUT, "stack kernel: a pipeline wait gave up after 2 s");
  }
  int64_t n = (int64_t)c.n_cand;
  int64_t sn = pow2_at_least(std::max<int64_t>(n, 1));
  L += launch_pad_keys(p->d_keys, p->d_idx, sn, p->d_ctr, p->s);
  L += launch_sort_gather(p->d_keys, p->d_idx, sn, p->d_ctr, p->d_cand, d_out, capacity, p->s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->s));
  p->launches = L;
  p->has_search = true;
  *h_count = n;
  if (n > capacity)
    return fail(ST_ERR_OVERFLOW, "%lld candidates exceed capacity %lld", (long long)n,
                (long long)capacity);
  return ST_OK;
}

// The refinement kernel over the fields' cubes of the last search.
st_status run_refine(st_plan_t* p, bool optimise, const float* theta, const int32_t* centre,
                     const int32_t* field, const st_candidate* cand, int64_t n, int steps,
                     int optimizer, float fwhm, float lr_pos, float lr_vel, float* J, float* snr,
                     float* grad, st_refined* out) {
  const int nf = (int)p->F.size();
  std::vector<FieldDev> h(nf);
  for (int fi = 0; fi < nf; ++fi)
    h[fi] = field_dev(p->F[fi], p->F[fi].last_frames, fi, p->o.storage);
  CK(cudaMemsetAsync(p->d_rerr, 0, sizeof(int), p->s));
  int l = launch_refine(h.data(), nf, p->d_fds, p->d_maps, p->d_times, p->d_tref, p->d_grid,
                        h[0].storage, optimise, theta, centre, field, cand, n, steps, optimizer,
                        fwhm, lr_pos, lr_vel, J, snr, grad, out, p->d_rerr, p->s);
  if (l < 0)
    return fail(ST_ERR_UNSUPPORTED, "refinement needs frame rows of a multiple of 16 bytes "
                "and at most %d frames per field", refine_max_frames());
  CK(cudaGetLastError());
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, p->d_rerr, sizeof(int), cudaMemcpyDeviceToHost, p->s));
  CK(cudaStreamSynchronize(p->s));
  p->launches = l;
  if (herr) return fail(ST_ERR_TIMEOUT, "refinement: a frame copy did not land within 2 s");
  return ST_OK;
}

}  // namespace

extern "C" {

int32_t st_version(void) { return ST_VERSION_MAJOR * 100 + ST_VERSION_MINOR; }

const char* st_last_error(void) { return g_err.c_str(); }

st_status st_plan(const st_field* fields, int32_t n_fields, const st_opts* opts,
                  void* cuda_stream, st_plan_t** out) {
  if (!out) return fail(ST_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!fields || n_fields <= 0 || n_fields > 255)
    return fail(ST_ERR_INVALID, "n_fields must be in [1, 255] and fields non-NULL");
  if (!opts) return fail(ST_ERR_INVALID, "opts is NULL");
  if (opts->storage < ST_F32 || opts->storage > ST_BF16)
    return fail(ST_ERR_INVALID, "storage must be ST_F32, ST_F16 or ST_BF16");
  if (opts->mode != ST_NEAREST && opts->mode != ST_BILINEAR)
    return fail(ST_ERR_INVALID, "mode must be ST_NEAREST or ST_BILINEAR");
  if (!std::isfinite(opts->cr_clip) || opts->cr_clip < 0.0f)
    return fail(ST_ERR_INVALID, "cr_clip must be finite and >= 0");
  if (opts->tile < -1 || opts->tile > 1 + fast_num_variants())
    return fail(ST_ERR_INVALID, "tile must be -1 (autotune), 0 (default), 1 (direct-gather "
                "kernel) or 2..%d (register-window variants)", 1 + fast_num_variants());
  if (opts->pending_capacity < 0 || opts->pending_capacity > (1ll << 31))
    return fail(ST_ERR_INVALID, "pending_capacity must be in [0, 2^31]");
  for (int i = 0; i < n_fields; ++i) {
    st_status st = validate_field(fields[i], i);
    if (st != ST_OK) return st;
  }
  st_plan_t* p = new (std::nothrow) st_plan_s();
  if (!p) return fail(ST_ERR_OOM, "host allocation failed");
  p->o = *opts;
  p->s = (cudaStream_t)cuda_stream;
  st_status st = ST_OK;
  auto guard = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == ST_OK)
      st = fail(e == cudaErrorMemoryAllocation ? ST_ERR_OOM : ST_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
    return e == cudaSuccess;
  };
  guard(cudaGetDevice(&p->device), "cudaGetDevice");
  guard(cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device),
        "cudaDeviceGetAttribute");
  if (opts->tune_cache) p->tune_cache = opts->tune_cache;
  p->F.resize(n_fields);
  int maxN = 0;
  for (int i = 0; i < n_fields && st == ST_OK; ++i) {
    FieldPlan& fp = p->F[i];
    fp.f = fields[i];
    const st_field& f = fp.f;
    maxN = std::max(maxN, f.n_frames);
    fp.nmin = f.min_coverage > 0 ? f.min_coverage : (f.n_frames + 1) / 2;
    guard(cudaMalloc(&fp.d_t, sizeof(double) * f.n_frames), "cudaMalloc(times)");
    guard(cudaMalloc(&fp.d_sx, sizeof(int32_t) * f.n_frames * (size_t)f.nvx), "cudaMalloc(sx)");
    guard(cudaMalloc(&fp.d_sy, sizeof(int32_t) * f.n_frames * (size_t)f.nvy), "cudaMalloc(sy)");
    guard(cudaMalloc(&fp.d_fx, sizeof(float) * f.n_frames * (size_t)f.nvx), "cudaMalloc(fx)");
    guard(cudaMalloc(&fp.d_fy, sizeof(float) * f.n_frames * (size_t)f.nvy), "cudaMalloc(fy)");
    // threshold and 1/sqrt tables, FP64 formulas rounded once to FP32
    std::vector<float> thr(f.n_frames + 1), rsq(f.n_frames + 1);
    for (int n = 0; n <= f.n_frames; ++n) {
      thr[n] = (float)((double)f.snr_threshold * std::sqrt((double)n));
      rsq[n] = n > 0 ? (float)(1.0 / std::sqrt((double)n)) : 0.0f;
    }
    if (guard(cudaMalloc(&fp.d_thr, sizeof(float) * (f.n_frames + 1)), "cudaMalloc(thr)"))
      guard(cudaMemcpy(fp.d_thr, thr.data(), sizeof(float) * thr.size(), cudaMemcpyHostToDevice),
            "cudaMemcpy(thr)");
    if (guard(cudaMalloc(&fp.d_rsq, sizeof(float) * (f.n_frames + 1)), "cudaMalloc(rsq)"))
      guard(cudaMemcpy(fp.d_rsq, rsq.data(), sizeof(float) * rsq.size(), cudaMemcpyHostToDevice),
            "cudaMemcpy(rsq)");
    if (opts->normalize || opts->storage != ST_F32)
      guard(cudaMalloc(&fp.d_cube, store_bytes(opts->storage) * (size_t)f.n_frames * fp.P()),
            "cudaMalloc(cube)");
    if (st == ST_OK && opts->tile != 1) {
      FieldDev probe = field_dev(fp, nullptr, i, opts->storage);
      if (fast_eligible(probe, opts->mode) && !fast_plan_build(probe, opts->mode, &fp.fast))
        st = fail(ST_ERR_OOM, "field %d: fast-kernel tables could not be allocated", i);
      if (fp.fast && opts->tile >= 2) fast_set_variant(fp.fast, opts->tile - 2);
    }
  }
  if (st == ST_OK) {
    p->pend_cap = opts->pending_capacity > 0 ? opts->pending_capacity : (4ll << 20);
    p->sort_cap = pow2_at_least(p->pend_cap);
    guard(cudaMalloc(&p->d_pend, sizeof(Pending) * p->pend_cap), "cudaMalloc(pending)");
    guard(cudaMalloc(&p->d_cand, sizeof(st_candidate) * p->pend_cap), "cudaMalloc(candidates)");
    guard(cudaMalloc(&p->d_keys, sizeof(uint64_t) * p->sort_cap), "cudaMalloc(keys)");
    guard(cudaMalloc(&p->d_idx, sizeof(uint32_t) * p->sort_cap), "cudaMalloc(idx)");
    guard(cudaMalloc(&p->d_ctr, sizeof(Counters)), "cudaMalloc(counters)");
    guard(cudaMallocHost(&p->h_ctr, sizeof(Counters)), "cudaMallocHost(counters)");
    guard(cudaMalloc(&p->d_fds, sizeof(FieldDev) * n_fields), "cudaMalloc(fields)");
    guard(cudaMalloc(&p->d_times, sizeof(double*) * n_fields), "cudaMalloc(times)");
    guard(cudaMalloc(&p->d_tref, sizeof(double) * n_fields), "cudaMalloc(tref)");
    guard(cudaMalloc(&p->d_grid, sizeof(double) * 4 * n_fields), "cudaMalloc(grid)");
    guard(cudaMalloc(&p->d_maps, sizeof(CUtensorMap) * n_fields), "cudaMalloc(maps)");
    guard(cudaMalloc(&p->d_rerr, sizeof(int)), "cudaMalloc(rerr)");
    if (st == ST_OK) {
      std::vector<double*> tp(n_fields);
      std::vector<double> tr(n_fields), gr(4 * n_fields);
      for (int i = 0; i < n_fields; ++i) {
        tp[i] = p->F[i].d_t;
        tr[i] = p->F[i].f.t_ref;
        gr[4 * i] = p->F[i].f.vx0;
        gr[4 * i + 1] = p->F[i].f.dvx;
        gr[4 * i + 2] = p->F[i].f.vy0;
        gr[4 * i + 3] = p->F[i].f.dvy;
      }
      guard(cudaMemcpy(p->d_times, tp.data(), sizeof(double*) * n_fields, cudaMemcpyHostToDevice),
            "cudaMemcpy(times)");
      guard(cudaMemcpy(p->d_tref, tr.data(), sizeof(double) * n_fields, cudaMemcpyHostToDevice),
            "cudaMemcpy(tref)");
      guard(cudaMemcpy(p->d_grid, gr.data(), sizeof(double) * 4 * n_fields, cudaMemcpyHostToDevice),
            "cudaMemcpy(grid)");
    }
    guard(cudaMalloc(&p->d_sky, sizeof(double) * sky_partial_doubles(maxN)), "cudaMalloc(sky)");
    guard(cudaEventCreate(&p->e0), "cudaEventCreate");
    guard(cudaEventCreate(&p->e1), "cudaEventCreate");
  }
  if (st != ST_OK) {
    free_plan(p);
    return st;
  }
  *out = p;
  return ST_OK;
}

void st_free(st_plan_t* plan) { free_plan(plan); }

st_status st_stack_search(st_plan_t* p, const float* const* d_frames, const double* const* h_times,
                          st_candidate* d_out, int64_t capacity, int64_t* h_count) {
  if (!p) return fail(ST_ERR_INVALID, "plan is NULL");
  return device_search(p, d_frames, h_times, d_out, capacity, h_count);
}

st_status st_stack_search_host(st_plan_t* p, const float* const* h_frames,
                               const double* const* h_times, st_candidate* h_out,
                               int64_t capacity, int64_t* h_count) {
  if (!p) return fail(ST_ERR_INVALID, "plan is NULL");
  if (!h_frames || !h_times || !h_count) return fail(ST_ERR_INVALID, "NULL argument");
  if (capacity < 0 || (capacity > 0 && !h_out))
    return fail(ST_ERR_INVALID, "capacity must be >= 0 and h_out non-NULL when capacity > 0");
  int nf = (int)p->F.size();
  std::vector<const float*> dptr(nf);
  for (int fi = 0; fi < nf; ++fi) {
    FieldPlan& fp = p->F[fi];
    if (!h_frames[fi]) return fail(ST_ERR_INVALID, "field %d: frames are NULL", fi);
    size_t bytes = sizeof(float) * (size_t)fp.f.n_frames * fp.P();
    if (!fp.d_frames_copy) CK(cudaMalloc(&fp.d_frames_copy, bytes));
    CK(cudaMemcpyAsync(fp.d_frames_copy, h_frames[fi], bytes, cudaMemcpyHostToDevice, p->s));
    dptr[fi] = fp.d_frames_copy;
  }
  if (capacity > p->hout_cap) {
    cudaFree(p->d_hout);
    p->d_hout = nullptr;
    p->hout_cap = 0;
    CK(cudaMalloc(&p->d_hout, sizeof(st_candidate) * capacity));
    p->hout_cap = capacity;
  }
  st_status st = device_search(p, dptr.data(), h_times, p->d_hout, capacity, h_count);
  if (st != ST_OK && st != ST_ERR_OVERFLOW) return st;
  int64_t n = std::min<int64_t>(*h_count < 0 ? 0 : *h_count, capacity);
  if (n > 0) {
    CK(cudaMemcpyAsync(h_out, p->d_hout, sizeof(st_candidate) * n, cudaMemcpyDeviceToHost, p->s));
    CK(cudaStreamSynchronize(p->s));
  }
  return st;
}

st_status st_shift_tables(st_plan_t* p, int32_t field, const double* h_times, int32_t* h_sx,
                          int32_t* h_sy, float* h_fx, float* h_fy) {
  if (!p) return fail(ST_ERR_INVALID, "plan is NULL");
  if (field < 0 || field >= (int)p->F.size()) return fail(ST_ERR_INVALID, "field out of range");
  if (!h_sx || !h_sy) return fail(ST_ERR_INVALID, "NULL table pointer");
  FieldPlan& fp = p->F[field];
  const st_field& f = fp.f;
  st_status st = check_times(h_times, f.n_frames, f, field);
  if (st != ST_OK) return st;
  // the field's tables now hold these timestamps' shifts: rebuild on the next search
  fp.tables_valid = false;
  ++p->gen;
  CK(cudaMemcpyAsync(fp.d_t, h_times, sizeof(double) * f.n_frames, cudaMemcpyHostToDevice, p->s));
  launch_shift_tables(fp.d_t, f.n_frames, f.t_ref, f.vx0, f.dvx, f.nvx, f.vy0, f.dvy, f.nvy,
                      p->o.mode, fp.d_sx, fp.d_sy, fp.d_fx, fp.d_fy, p->s);
  CK(cudaGetLastError());
  size_t nx = (size_t)f.n_frames * f.nvx, ny = (size_t)f.n_frames * f.nvy;
  CK(cudaMemcpyAsync(h_sx, fp.d_sx, sizeof(int32_t) * nx, cudaMemcpyDeviceToHost, p->s));
  CK(cudaMemcpyAsync(h_sy, fp.d_sy, sizeof(int32_t) * ny, cudaMemcpyDeviceToHost, p->s));
  if (h_fx) CK(cudaMemcpyAsync(h_fx, fp.d_fx, sizeof(float) * nx, cudaMemcpyDeviceToHost, p->s));
  if (h_fy) CK(cudaMemcpyAsync(h_fy, fp.d_fy, sizeof(float) * ny, cudaMemcpyDeviceToHost, p->s));
  CK(cudaStreamSynchronize(p->s));
  return ST_OK;
}

st_status st_normalize(st_plan_t* p, int32_t field, const float* d_frames, void* d_cube,
                       double* h_mu, double* h_sigma) {
  if (!p) return fail(ST_ERR_INVALID, "plan is NULL");
  if (field < 0 || field >= (int)p->F.size()) return fail(ST_ERR_INVALID, "field out of range");
  if (!d_frames || !d_cube) return fail(ST_ERR_INVALID, "NULL frames or cube");
  FieldPlan& fp = p->F[field];
  const st_field& f = fp.f;
  double* d_ms = nullptr;
  CK(cudaMalloc(&d_ms, sizeof(double) * 2 * f.n_frames));
  launch_normalize(d_frames, f.n_frames, fp.P(), 1, p->o.cr_clip, p->o.storage, d_cube, d_ms,
                   d_ms + f.n_frames, p->d_sky, p->s);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && h_mu)
    e = cudaMemcpyAsync(h_mu, d_ms, sizeof(double) * f.n_frames, cudaMemcpyDeviceToHost, p->s);
  if (e == cudaSuccess && h_sigma)
    e = cudaMemcpyAsync(h_sigma, d_ms + f.n_frames, sizeof(double) * f.n_frames,
                        cudaMemcpyDeviceToHost, p->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->s);
  cudaFree(d_ms);
  if (e != cudaSuccess) return fail(ST_ERR_CUDA, "st_normalize: %s", cudaGetErrorString(e));
  return ST_OK;
}

st_status st_dump_stack(st_plan_t* p, int32_t field, const float* d_frames, const double* h_times,
                        const int32_t* h_k, int32_t n_k, float* d_S, int32_t* d_ncov) {
  if (!p) return fail(ST_ERR_INVALID, "plan is NULL");
  if (field < 0 || field >= (int)p->F.size()) return fail(ST_ERR_INVALID, "field out of range");
  if (!d_frames || !h_times || !h_k || n_k <= 0 || !d_S)
    return fail(ST_ERR_INVALID, "NULL argument or n_k <= 0");
  FieldPlan& fp = p->F[field];
  for (int q = 0; q < n_k; ++q)
    if (h_k[q] < 0 || h_k[q] >= fp.nk()) return fail(ST_ERR_INVALID, "velocity index out of range");
  int64_t L = 0;
  st_status st = prepare_field(p, field, d_frames, h_times, &L);
  if (st != ST_OK) return st;
  int32_t* d_k = nullptr;
  CK(cudaMalloc(&d_k, sizeof(int32_t) * n_k));
  cudaError_t e = cudaMemcpyAsync(d_k, h_k, sizeof(int32_t) * n_k, cudaMemcpyHostToDevice, p->s);
  FieldDev fd = field_dev(fp, d_frames, field, p->o.storage);
  bool whole = n_k == fp.nk();
  for (int q = 0; q < n_k && whole; ++q) whole = h_k[q] == q;
  if (e == cudaSuccess) {
    int n = -1;
    if (whole && fp.fast) {
      bool fits = false;
      fast_prepare(fd, fp.fast, p->s, &fits);
      if (fits)
        n = launch_stack_fast(fd, fp.fast, 0, n_k, nullptr, d_S, d_ncov, p->d_pend, p->pend_cap,
                              p->d_ctr, p->s);
    }
    if (n < 0)
      launch_stack_generic(fd, p->o.mode, 0, n_k, d_k, d_S, d_ncov, p->d_pend, p->pend_cap,
                           p->d_ctr, p->s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->s);
  cudaFree(d_k);
  if (e != cudaSuccess) return fail(ST_ERR_CUDA, "st_dump_stack: %s", cudaGetErrorString(e));
  return ST_OK;
}

int64_t st_last_launch_count(const st_plan_t* p) { return p ? p->launches : 0; }

int32_t st_last_graph_replayed(const st_plan_t* p) { return p && p->last_replayed ? 1 : 0; }

st_status st_link_tracks(st_plan_t* p, const st_candidate* d_cand, int64_t n, int32_t r_xy,
                         int32_t r_v, st_track* d_tracks, int64_t capacity, int64_t* h_count) {
  if (!p || !h_count) return fail(ST_ERR_INVALID, "NULL argument");
  *h_count = 0;
  if (n < 0 || (n > 0 && !d_cand) || capacity < 0 || (capacity > 0 && !d_tracks))
    return fail(ST_ERR_INVALID, "n, capacity >= 0 and non-NULL buffers required");
  if (r_xy < 0 || r_v < 0) return fail(ST_ERR_INVALID, "r_xy and r_v must be >= 0");
  if (n > 0x7fffffffll) return fail(ST_ERR_UNSUPPORTED, "at most 2^31 - 1 detections");
  if (!p->has_search) return fail(ST_ERR_INVALID, "st_link_tracks needs a prior st_stack_search");
  if (n == 0) return ST_OK;
  const int64_t need = link_workspace_bytes(n);
  if (need > p->link_ws_bytes) {
    cudaFree(p->d_link_ws);
    p->d_link_ws = nullptr;
    p->link_ws_bytes = 0;
    CK(cudaMalloc(&p->d_link_ws, need));
    p->link_ws_bytes = need;
  }
  int64_t nt = 0;
  int l = launch_link_tracks(d_cand, n, p->d_fds, p->d_grid, r_xy, r_v, p->d_link_ws, d_tracks,
                             capacity, &nt, p->s);
  CK(cudaGetLastError());
  if (l < 0) return fail(ST_ERR_CUDA, "track linking failed");
  p->launches = l;
  *h_count = nt;
  if (nt > capacity)
    return fail(ST_ERR_OVERFLOW, "%lld tracks exceed capacity %lld", (long long)nt,
                (long long)capacity);
  return ST_OK;
}

static bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + nb && y < x + na;
}

st_status st_median_subtract(const float* d_in, int32_t n_frames, int32_t height, int32_t width,
                             float* d_out, float* d_median, void* cuda_stream) {
  if (!d_in || !d_out) return fail(ST_ERR_INVALID, "NULL frames");
  if (n_frames <= 0 || height <= 0 || width <= 0)
    return fail(ST_ERR_INVALID, "n_frames, height and width must be > 0");
  if (n_frames > median_max_frames())
    return fail(ST_ERR_UNSUPPORTED, "median over at most %d frames (got %d)",
                median_max_frames(), n_frames);
  const int64_t P = (int64_t)height * width;
  if (launch_median_subtract(d_in, n_frames, P, d_out, d_median, (cudaStream_t)cuda_stream) < 0)
    return fail(ST_ERR_INVALID, "frame too large for the median kernel's grid");
  CK(cudaGetLastError());
  return ST_OK;
}

st_status st_sum_frames(const float* d_in, int32_t n_frames, int32_t height, int32_t width,
                        int32_t n_sum, const double* h_times, float* d_out, double* h_times_out,
                        void* cuda_stream) {
  if (!d_in || !d_out) return fail(ST_ERR_INVALID, "NULL frames");
  if (n_frames <= 0 || height <= 0 || width <= 0 || n_sum <= 0)
    return fail(ST_ERR_INVALID, "n_frames, height, width and n_sum must be > 0");
  if (h_times_out && !h_times) return fail(ST_ERR_INVALID, "h_times_out needs h_times");
  const int64_t P = (int64_t)height * width;
  const int M = n_frames / n_sum;
  if (overlaps(d_in, sizeof(float) * P * n_frames, d_out, sizeof(float) * P * (M > 0 ? M : 0)))
    return fail(ST_ERR_INVALID, "d_out overlaps d_in");
  if (launch_sum_frames(d_in, n_sum, M, P, d_out, (cudaStream_t)cuda_stream) < 0)
    return fail(ST_ERR_INVALID, "sizes exceed the sum kernel's grid");
  CK(cudaGetLastError());
  if (h_times_out)
    for (int m = 0; m < M; ++m) {
      double ts = 0.0;
      for (int i = m * n_sum; i < (m + 1) * n_sum; ++i) ts += h_times[i];
      h_times_out[m] = ts / n_sum;
    }
  return ST_OK;
}

st_status st_bin2x2(const float* d_in, int32_t n_frames, int32_t height, int32_t width,
                    float* d_out, void* cuda_stream) {
  if (!d_in || !d_out) return fail(ST_ERR_INVALID, "NULL frames");
  if (n_frames <= 0 || height <= 0 || width <= 0)
    return fail(ST_ERR_INVALID, "n_frames, height and width must be > 0");
  const size_t nin = sizeof(float) * (size_t)n_frames * height * width;
  const size_t nout = sizeof(float) * (size_t)n_frames * (height / 2) * (width / 2);
  if (overlaps(d_in, nin, d_out, nout)) return fail(ST_ERR_INVALID, "d_out overlaps d_in");
  if (launch_bin2x2(d_in, n_frames, height, width, d_out, (cudaStream_t)cuda_stream) < 0)
    return fail(ST_ERR_INVALID, "sizes exceed the binning kernel's grid");
  CK(cudaGetLastError());
  return ST_OK;
}

int32_t st_last_stack_variant(const st_plan_t* p, int32_t field) {
  if (!p || field < 0 || field >= (int)p->F.size()) return -1;
  return p->F[field].last_variant;
}

const char* st_stack_variant_name(const st_plan_t* p, int32_t field) {
  if (!p || field < 0 || field >= (int)p->F.size()) return "?";
  const FieldPlan& fp = p->F[field];
  if (fp.last_variant == 0) return "direct-gather";
  if (fp.last_variant != 1 || !fp.fast) return "?";
  return fast_variant_name(fp.fast, p->o.storage);
}

st_status st_last_stack_kernel_time(const st_plan_t* p, double* ms, int64_t* launches) {
  if (!p || !ms || !launches) return fail(ST_ERR_INVALID, "NULL argument");
  *ms = p->stack_ms;
  *launches = p->stack_launches;
  return ST_OK;
}

st_status st_refine(st_plan_t* p, const st_candidate* d_in, int64_t n, int32_t steps,
                    int32_t optimizer, float fwhm, float lr_pos, float lr_vel, st_refined* d_out,
                    float* d_grad_out) {
  if (!p) return fail(ST_ERR_INVALID, "plan is NULL");
  if (n < 0 || (n > 0 && (!d_in || !d_out)) || steps < 0 || steps > 100000)
    return fail(ST_ERR_INVALID, "n >= 0, d_in/d_out non-NULL, 0 <= steps <= 100000");
  if (!(fwhm > 0.0f) || !std::isfinite(fwhm) || !std::isfinite(lr_pos) || !std::isfinite(lr_vel))
    return fail(ST_ERR_INVALID, "fwhm > 0 and finite learning rates required");
  if (optimizer != 0 && optimizer != 1)
    return fail(ST_ERR_INVALID, "optimizer must be 0 (Adam) or 1 (Gauss-Newton)");
  if (optimizer == 1 && !(lr_pos >= 0.0f))
    return fail(ST_ERR_INVALID, "Gauss-Newton damping (lr_pos) must be >= 0");
  if (n > 0x7fffffffll) return fail(ST_ERR_UNSUPPORTED, "at most 2^31 - 1 candidates per call");
  if (!p->has_search) return fail(ST_ERR_INVALID, "st_refine needs a prior st_stack_search");
  if (n == 0) return ST_OK;
  return run_refine(p, true, nullptr, nullptr, nullptr, d_in, n, steps, optimizer, fwhm, lr_pos,
                    lr_vel, nullptr, nullptr, d_grad_out, d_out);
}

st_status st_refine_eval(st_plan_t* p, const float* d_theta, const int32_t* d_centre,
                         const int32_t* d_field, int64_t n, float fwhm, float* d_J, float* d_snr,
                         float* d_grad) {
  if (!p) return fail(ST_ERR_INVALID, "plan is NULL");
  if (n < 0 || (n > 0 && (!d_theta || !d_centre || !d_field || !d_J || !d_snr)))
    return fail(ST_ERR_INVALID, "n >= 0 and theta, centre, field, J, snr non-NULL");
  if (!(fwhm > 0.0f) || !std::isfinite(fwhm)) return fail(ST_ERR_INVALID, "fwhm must be > 0");
  if (n > 0x7fffffffll) return fail(ST_ERR_UNSUPPORTED, "at most 2^31 - 1 candidates per call");
  if (!p->has_search) return fail(ST_ERR_INVALID, "st_refine_eval needs a prior st_stack_search");
  if (n == 0) return ST_OK;
  return run_refine(p, false, d_theta, d_centre, d_field, nullptr, n, 0, 0, fwhm, 0.0f, 0.0f,
                    d_J, d_snr, d_grad, nullptr);
}

}  // extern "C"
