"""Python binding of the GB300 synthetic-tracking library (include/st.h).

Argument marshalling only: every step of the search runs in the CUDA kernels
of ``libst.so``.  PyTorch provides device memory and streams.  There is no CPU
fallback: importing this package without the built library raises.

The method is the synthetic-tracking (shift-and-stack) search of Burdanov,
Hasler & de Wit (2023), Sec. 1 and Sec. 2.1.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libst.so")

ST_OK, ST_ERR_INVALID, ST_ERR_CUDA, ST_ERR_OOM, ST_ERR_OVERFLOW, ST_ERR_TIMEOUT, \
    ST_ERR_UNSUPPORTED = range(7)
STATUS_NAMES = ["ST_OK", "ST_ERR_INVALID", "ST_ERR_CUDA", "ST_ERR_OOM", "ST_ERR_OVERFLOW",
                "ST_ERR_TIMEOUT", "ST_ERR_UNSUPPORTED"]
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
MODE = {"nearest": 0, "bilinear": 1}

CAND_DTYPE = np.dtype([("x", np.int32), ("y", np.int32), ("k", np.int32), ("field", np.int32),
                       ("stack", np.float32), ("snr", np.float32), ("n_cov", np.int32)])
TRACK_DTYPE = np.dtype([("x", np.int32), ("y", np.int32), ("k", np.int32), ("field", np.int32),
                        ("stack", np.float32), ("snr", np.float32), ("n_cov", np.int32),
                        ("members", np.int32), ("vx", np.float32), ("vy", np.float32),
                        ("speed", np.float32), ("pa", np.float32)])
REFINED_DTYPE = np.dtype([("vx", np.float32), ("vy", np.float32), ("x0", np.float32),
                          ("y0", np.float32), ("flux", np.float32), ("snr", np.float32),
                          ("obj", np.float32), ("field", np.int32)])


class StError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class Field(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("n_frames", C.c_int32),
                ("t_ref", C.c_double), ("vx0", C.c_double), ("dvx", C.c_double),
                ("nvx", C.c_int32), ("vy0", C.c_double), ("dvy", C.c_double),
                ("nvy", C.c_int32), ("snr_threshold", C.c_float), ("min_coverage", C.c_int32)]


class Opts(C.Structure):
    _fields_ = [("storage", C.c_int), ("mode", C.c_int), ("normalize", C.c_int32),
                ("cr_clip", C.c_float), ("use_graph", C.c_int32), ("tile", C.c_int32),
                ("tune_cache", C.c_char_p), ("pending_capacity", C.c_int64)]


_lib = None


def lib():
    """The loaded libst.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libst.so not built at {LIB_PATH}: run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.st_version.restype = C.c_int32
        L.st_last_error.restype = C.c_char_p
        L.st_plan.argtypes = [P, C.c_int32, P, P, P]
        L.st_free.argtypes = [P]
        L.st_free.restype = None
        L.st_stack_search.argtypes = [P, P, P, P, C.c_int64, P]
        L.st_stack_search_host.argtypes = [P, P, P, P, C.c_int64, P]
        L.st_refine.argtypes = [P, P, C.c_int64, C.c_int32, C.c_int32, C.c_float, C.c_float,
                                C.c_float, P, P]
        L.st_refine_eval.argtypes = [P, P, P, P, C.c_int64, C.c_float, P, P, P]
        L.st_shift_tables.argtypes = [P, C.c_int32, P, P, P, P, P]
        L.st_normalize.argtypes = [P, C.c_int32, P, P, P, P]
        L.st_dump_stack.argtypes = [P, C.c_int32, P, P, P, C.c_int32, P, P]
        L.st_last_launch_count.argtypes = [P]
        L.st_last_launch_count.restype = C.c_int64
        L.st_last_stack_kernel_time.argtypes = [P, P, P]
        L.st_last_stack_variant.argtypes = [P, C.c_int32]
        L.st_last_stack_variant.restype = C.c_int32
        L.st_stack_variant_name.argtypes = [P, C.c_int32]
        L.st_stack_variant_name.restype = C.c_char_p
        L.st_last_graph_replayed.argtypes = [P]
        L.st_last_graph_replayed.restype = C.c_int32
        L.st_probe_add_rate.argtypes = [C.c_int32, C.c_int32, P, P]
        _lib = L
    return _lib


def _check(status):
    if status != ST_OK:
        raise StError(status, lib().st_last_error().decode())


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_field(d):
    """st_field from a dict with the keys of synth.field_params."""
    return Field(int(d["width"]), int(d["height"]), int(d["n_frames"]), float(d["t_ref"]),
                 float(d["vx0"]), float(d["dvx"]), int(d["nvx"]), float(d["vy0"]),
                 float(d["dvy"]), int(d["nvy"]), float(d["snr_threshold"]),
                 int(d.get("min_coverage", 0)))


class Plan:
    """A search plan over one or more fields (st_plan / st_free)."""

    def __init__(self, fields, storage="f32", mode="nearest", normalize=False, cr_clip=0.0,
                 use_graph=False, tile=0, tune_cache=None, pending_capacity=0, stream=None):
        if isinstance(fields, dict):
            fields = [fields]
        self.fields = [dict(f) for f in fields]
        arr = (Field * len(fields))(*[make_field(f) for f in fields])
        self._tc = tune_cache.encode() if tune_cache else None
        opts = Opts(STORAGE[storage], MODE[mode], int(bool(normalize)), float(cr_clip),
                    int(bool(use_graph)), int(tile), self._tc, int(pending_capacity))
        self._opts = opts
        self.storage, self.mode = storage, mode
        self._stream = stream
        h = C.c_void_p()
        _check(lib().st_plan(C.cast(arr, C.c_void_p), len(fields), C.byref(opts),
                             _stream_handle(stream), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().st_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- search
    def search(self, frames, times, capacity=1 << 20, out=None):
        """st_stack_search.  frames: list of CUDA float32 tensors [N][H][W];
        times: list of float64 arrays.  Returns (out tensor [capacity, 7] int32
        on the device, total count)."""
        import torch
        frames = [frames] if hasattr(frames, "data_ptr") else list(frames)
        times = [times] if isinstance(times, np.ndarray) and times.ndim == 1 else list(times)
        for f in frames:
            if not (f.is_cuda and f.dtype == torch.float32 and f.is_contiguous()):
                raise ValueError("frames must be contiguous CUDA float32 tensors")
        tarr = [np.ascontiguousarray(t, np.float64) for t in times]
        fptr = (C.c_void_p * len(frames))(*[f.data_ptr() for f in frames])
        tptr = (C.c_void_p * len(tarr))(*[t.ctypes.data for t in tarr])
        if out is None:
            out = torch.empty((max(capacity, 1), 7), dtype=torch.int32, device=frames[0].device)
        cnt = C.c_int64()
        st = lib().st_stack_search(self._h, C.cast(fptr, C.c_void_p), C.cast(tptr, C.c_void_p),
                                   _ptr(out), capacity, C.byref(cnt))
        if st not in (ST_OK, ST_ERR_OVERFLOW) or cnt.value < 0:
            _check(st)
        return out, cnt.value, st

    def search_host(self, frames, times, capacity=1 << 20):
        """st_stack_search_host with host numpy frames; returns the structured
        candidate array (numpy) and the total count."""
        frames = [frames] if isinstance(frames, np.ndarray) and frames.ndim == 3 else list(frames)
        times = [times] if isinstance(times, np.ndarray) and times.ndim == 1 else list(times)
        fr = [np.ascontiguousarray(f, np.float32) for f in frames]
        tarr = [np.ascontiguousarray(t, np.float64) for t in times]
        fptr = (C.c_void_p * len(fr))(*[f.ctypes.data for f in fr])
        tptr = (C.c_void_p * len(tarr))(*[t.ctypes.data for t in tarr])
        out = np.zeros(max(capacity, 1), CAND_DTYPE)
        cnt = C.c_int64()
        st = lib().st_stack_search_host(self._h, C.cast(fptr, C.c_void_p),
                                        C.cast(tptr, C.c_void_p), _np_ptr(out), capacity,
                                        C.byref(cnt))
        if st not in (ST_OK, ST_ERR_OVERFLOW) or cnt.value < 0:
            _check(st)
        return out[:min(cnt.value, capacity)], cnt.value

    @staticmethod
    def to_numpy(out, count):
        n = min(count, out.shape[0])
        return out[:n].cpu().numpy().view(CAND_DTYPE).reshape(-1)

    def candidates(self, frames, times, capacity=1 << 20):
        out, n, st = self.search(frames, times, capacity)
        if st == ST_ERR_OVERFLOW:
            out, n, st = self.search(frames, times, n)
        return self.to_numpy(out, n)

    # ----------------------------------------------------------- diagnostics
    def shift_tables(self, field, times):
        f = self.fields[field]
        N = int(f["n_frames"])
        sx = np.zeros((N, f["nvx"]), np.int32)
        sy = np.zeros((N, f["nvy"]), np.int32)
        fx = np.zeros((N, f["nvx"]), np.float32)
        fy = np.zeros((N, f["nvy"]), np.float32)
        t = np.ascontiguousarray(times, np.float64)
        _check(lib().st_shift_tables(self._h, field, _np_ptr(t), _np_ptr(sx), _np_ptr(sy),
                                     _np_ptr(fx), _np_ptr(fy)))
        return sx, sy, fx, fy

    def normalize(self, field, frames):
        import torch
        N, H, W = frames.shape
        dt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[self.storage]
        cube = torch.empty((N, H, W), dtype=dt, device=frames.device)
        mu = np.zeros(N)
        sd = np.zeros(N)
        _check(lib().st_normalize(self._h, field, _ptr(frames), _ptr(cube), _np_ptr(mu),
                                  _np_ptr(sd)))
        return cube, mu, sd

    def dump_stack(self, field, frames, times, ks):
        import torch
        N, H, W = frames.shape
        ks = np.ascontiguousarray(ks, np.int32)
        S = torch.empty((ks.size, H, W), dtype=torch.float32, device=frames.device)
        Cv = torch.empty((ks.size, H, W), dtype=torch.int32, device=frames.device)
        t = np.ascontiguousarray(times, np.float64)
        _check(lib().st_dump_stack(self._h, field, _ptr(frames), _np_ptr(t), _np_ptr(ks),
                                   ks.size, _ptr(S), _ptr(Cv)))
        return S, Cv

    # ------------------------------------------------------------ refinement
    def refine(self, cands, n=None, steps=20, fwhm=3.0, lr_pos=0.05, lr_vel=None, grad=False,
               optimizer="adam", damping=1.0):
        """st_refine: refinement of candidates (device tensor [n, 7] int32 as
        returned by search) by Adam (lr_pos, lr_vel) or Gauss-Newton
        (optimizer="gn", damping).  Returns the refined records (numpy) and,
        if grad, dJ/dtheta [n, 5] at the final parameters."""
        import torch
        n = cands.shape[0] if n is None else n
        if optimizer not in ("adam", "gn"):
            raise ValueError("optimizer must be 'adam' or 'gn'")
        opt = 1 if optimizer == "gn" else 0
        if opt == 1:
            lr_pos, lr_vel = damping, 0.0
        elif lr_vel is None:
            lr_vel = 0.05 * float(self.fields[0]["dvx"])
        out = torch.empty((max(n, 1), 8), dtype=torch.int32, device=cands.device)
        g = torch.empty((max(n, 1), 5), dtype=torch.float32, device=cands.device) if grad else None
        _check(lib().st_refine(self._h, _ptr(cands), n, steps, opt, fwhm, lr_pos, lr_vel,
                               _ptr(out), _ptr(g) if grad else None))
        rec = out[:n].cpu().numpy().view(REFINED_DTYPE).reshape(-1)
        return (rec, g[:n]) if grad else rec

    def link_tracks(self, cands, n=None, r_xy=2, r_v=1):
        """st_link_tracks: the detections (device tensor [n, 7] int32 in the
        order search returns them) linked into tracks; numpy TRACK_DTYPE."""
        import torch
        n = cands.shape[0] if n is None else n
        L = lib()
        L.st_link_tracks.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int32,
                                     C.c_void_p, C.c_int64, C.c_void_p]
        out = torch.empty((max(n, 1), 12), dtype=torch.int32, device=cands.device)
        cnt = C.c_int64()
        _check(L.st_link_tracks(self._h, _ptr(cands), n, r_xy, r_v, _ptr(out), max(n, 1),
                                C.byref(cnt)))
        return out[:cnt.value].cpu().numpy().view(TRACK_DTYPE).reshape(-1)

    def refine_eval(self, theta, centre, field=None, fwhm=3.0, grad=True):
        """st_refine_eval: J [n], SNR [n] and (optionally) dJ/dtheta [n, 5] at
        theta ([n, 5] float32 CUDA: vx, vy, x0, y0, F), cutout centres [n, 2]."""
        import torch
        theta = theta.detach().contiguous().float()
        n = theta.shape[0]
        dev_ = theta.device
        centre = torch.as_tensor(centre, dtype=torch.int32, device=dev_).contiguous()
        if field is None:
            field = torch.zeros(n, dtype=torch.int32, device=dev_)
        field = torch.as_tensor(field, dtype=torch.int32, device=dev_).contiguous()
        J = torch.empty(n, dtype=torch.float32, device=dev_)
        snr = torch.empty(n, dtype=torch.float32, device=dev_)
        g = torch.empty((n, 5), dtype=torch.float32, device=dev_) if grad else None
        _check(lib().st_refine_eval(self._h, _ptr(theta), _ptr(centre), _ptr(field), n, fwhm,
                                    _ptr(J), _ptr(snr), _ptr(g) if grad else None))
        return J, snr, g

    def stack_variant_name(self, field=0):
        """Name of the stack kernel variant field `field` used in the last search."""
        return lib().st_stack_variant_name(self._h, field).decode()

    def last_stack_variant(self, field=0):
        """1 if field used the register-window kernel in the last search, 0 if
        the direct-gather kernel, -1 before any search."""
        return lib().st_last_stack_variant(self._h, field)

    def last_graph_replayed(self):
        """True if the last search's device part ran as a CUDA graph."""
        return bool(lib().st_last_graph_replayed(self._h))

    def last_launch_count(self):
        return lib().st_last_launch_count(self._h)

    def last_stack_kernel_time(self):
        ms = C.c_double()
        n = C.c_int64()
        _check(lib().st_last_stack_kernel_time(self._h, C.byref(ms), C.byref(n)))
        return ms.value, n.value


def _refine_objective_class():
    import torch

    class RefineObjective(torch.autograd.Function):
        """J(theta) of the refinement on a plan's last searched frames.  The
        backward pass calls the library's hand-written adjoint, recomputing the
        shifted cutouts instead of storing them."""

        @staticmethod
        def forward(ctx, theta, plan, centre, field, fwhm):
            J, _, _ = plan.refine_eval(theta, centre, field, fwhm, grad=False)
            ctx.save_for_backward(theta.detach())
            ctx.plan, ctx.centre, ctx.field, ctx.fwhm = plan, centre, field, fwhm
            return J

        @staticmethod
        def backward(ctx, gJ):
            (theta,) = ctx.saved_tensors
            _, _, g = ctx.plan.refine_eval(theta, ctx.centre, ctx.field, ctx.fwhm, grad=True)
            return gJ[:, None] * g, None, None, None, None

    return RefineObjective


def refine_objective(theta, plan, centre, field=None, fwhm=3.0):
    """Differentiable J(theta) (torch.autograd) with the library's adjoint."""
    return _refine_objective_class().apply(theta, plan, centre, field, fwhm)


def probe_add_rate(variant=1, iters=20000):
    """FP32 add-rate microbenchmark: (adds per SM clock, T adds/s)."""
    a = C.c_double()
    t = C.c_double()
    _check(lib().st_probe_add_rate(variant, iters, C.byref(a), C.byref(t)))
    return a.value, t.value


def probe_wait_timeout(limit_us=100000):
    """st_probe_wait_timeout: (timed out?, microseconds waited) of a bounded
    wait on a phase that never completes."""
    L = lib()
    L.st_probe_wait_timeout.argtypes = [C.c_int32, C.c_void_p, C.c_void_p]
    flag = C.c_int32()
    us = C.c_double()
    _check(L.st_probe_wait_timeout(int(limit_us), C.byref(flag), C.byref(us)))
    return bool(flag.value), us.value


def search_noalloc(field, frames, times, capacity=1 << 16, mode="nearest", stream=None):
    """st_stack_search_noalloc: one-field search whose scratch lives in a fixed
    device array inside the library (for callers that cannot allocate device
    memory).  frames: contiguous CUDA float32 tensor [N][H][W].  Returns
    (out tensor [capacity, 7] int32, total count, status).  Calls that overlap
    on the GPU share the array and must be serialised."""
    import torch
    L = lib()
    L.st_stack_search_noalloc.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    if not (frames.is_cuda and frames.dtype == torch.float32 and frames.is_contiguous()):
        raise ValueError("frames must be a contiguous CUDA float32 tensor")
    f = make_field(field)
    t = np.ascontiguousarray(times, np.float64)
    out = torch.empty((max(capacity, 1), 7), dtype=torch.int32, device=frames.device)
    cnt = C.c_int64()
    status = L.st_stack_search_noalloc(C.byref(f), MODE[mode], _ptr(frames), _np_ptr(t),
                                       _ptr(out), capacity, C.byref(cnt), _stream_handle(stream))
    if status not in (ST_OK, ST_ERR_OVERFLOW) or cnt.value < 0:
        _check(status)
    return out, cnt.value, status


# ------------------------------------------------------ pre-tracking front end

def _cube(frames):
    import torch
    if not (frames.is_cuda and frames.dtype == torch.float32 and frames.is_contiguous() and
            frames.dim() == 3):
        raise ValueError("frames must be a contiguous CUDA float32 tensor [N][H][W]")
    return frames.shape


def median_subtract(frames, out=None, with_median=False, stream=None):
    """st_median_subtract: frames minus their per-pixel median over the frames
    (finite samples; Sec. 2.1 star removal).  out may be frames (in place).
    Returns out, or (out, median [H][W]) with with_median."""
    import torch
    N, H, W = _cube(frames)
    out = torch.empty_like(frames) if out is None else out
    med = torch.empty((H, W), dtype=torch.float32, device=frames.device) if with_median else None
    L = lib()
    L.st_median_subtract.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                     C.c_void_p, C.c_void_p]
    _check(L.st_median_subtract(_ptr(frames), N, H, W, _ptr(out),
                                _ptr(med) if with_median else None, _stream_handle(stream)))
    return (out, med) if with_median else out


def sum_frames(frames, times, n_sum, stream=None):
    """st_sum_frames: sums of every n_sum frames (a trailing partial group is
    dropped) and the mean time stamp of each group."""
    import torch
    N, H, W = _cube(frames)
    M = N // n_sum
    out = torch.empty((max(M, 1), H, W), dtype=torch.float32, device=frames.device)
    t = np.ascontiguousarray(times, np.float64)
    tout = np.zeros(max(M, 1), np.float64)
    L = lib()
    L.st_sum_frames.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    _check(L.st_sum_frames(_ptr(frames), N, H, W, int(n_sum), _np_ptr(t), _ptr(out),
                           _np_ptr(tout), _stream_handle(stream)))
    return out[:M], tout[:M]


def bin2x2(frames, stream=None):
    """st_bin2x2: 2 x 2 block sums [N][H/2][W/2]."""
    import torch
    N, H, W = _cube(frames)
    out = torch.empty((N, max(H // 2, 1), max(W // 2, 1)), dtype=torch.float32,
                      device=frames.device)
    L = lib()
    L.st_bin2x2.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                            C.c_void_p]
    _check(L.st_bin2x2(_ptr(frames), N, H, W, _ptr(out), _stream_handle(stream)))
    return out[:, :H // 2, :W // 2]


def version():
    return lib().st_version()
