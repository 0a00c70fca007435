"""Seeded synthetic fields: the inputs shared by the oracle and the CUDA library.

This module makes inputs only (noise, sky residuals, masked star blobs, cosmic
rays, movers on linear trajectories).  It holds none of the search's
arithmetic.  The heavy parts are in ``synth.c`` (counter-based Philox4x32-10,
OpenMP); the random choices of mover parameters use numpy's Philox generator.

The workload recipes stand in for the SPECULOOS data of the paper (2K x 2K
frames at 0.35"/px, Sec. 3), which is not available:

* ``tiny``      16 x 128^2, t_i = i, 3 integer movers, integer grid +-10 (441)
* ``mid``       64 x 1024^2, 2 h with +-5 s jitter, sky residual 0.1 sigma,
                200 NaN star blobs, 20 movers, grid +-40 px/h step 0.5 (161^2)
* ``speculoos`` 256 x 2048^2, 50 s cadence, cosmic rays 1e-5 /px/frame,
                100 movers at 0.5-100 px/h, grid +-100 px/h step 0.25 (801^2)
* ``batched``   24 fields: N in [40, 400], sizes {512, 1024, 2048}^2, baselines
                1-8 h, grid step 1 px over the baseline, +-60 px/h
* ``refine``    ``speculoos`` with 300 frames (the refinement workload)
* ``multinight`` 2 nights x 64 frames of 1024^2 (2 min cadence, nights 24 h
                apart), slow movers (<= 5 px/h), grid +-5 px/h with a step of
                1 px over the whole baseline (a large, sparse-in-time grid)
"""
import ctypes as C
import math
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libsynth.so")
BASE_SEED = 20230313
_lib = None


def build(force=False):
    src = os.path.join(HERE, "synth.c")
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(src):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
                    "-shared", "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.c_void_p
        L.synth_philox.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_int64, P]
        L.synth_normal.argtypes = [P, C.c_int64, C.c_uint64, C.c_uint64, C.c_float]
        L.synth_add_smooth_residual.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_uint64,
                                                C.c_int, C.c_float]
        L.synth_render_movers.argtypes = [P, C.c_int, C.c_int, C.c_int, P, C.c_double, P,
                                          C.c_int, C.c_double]
        L.synth_add_cosmics.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_double,
                                        C.c_double, C.c_double, P, C.c_int64]
        L.synth_add_cosmics.restype = C.c_int64
        L.synth_mask_blobs.argtypes = [P, C.c_int, C.c_int, C.c_int, P, C.c_int]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def philox_words(seed, stream, n_blocks, first=0):
    out = np.zeros(4 * n_blocks, np.uint32)
    lib().synth_philox(seed, stream, first, n_blocks, _p(out))
    return out


def noise(n_frames, height, width, seed, sigma=1.0, out=None):
    """Gaussian noise cube [N][H][W] float32; frame i uses Philox stream i."""
    if out is None:
        out = np.empty((n_frames, height, width), np.float32)
    P = height * width
    for i in range(n_frames):
        lib().synth_normal(_p(out[i]), P, seed, i, sigma)
    return out


def render_movers(frames, t, t_ref, movers, fwhm=3.0):
    movers = np.ascontiguousarray(movers, np.float64).reshape(-1, 5)
    t = np.ascontiguousarray(t, np.float64)
    N, H, W = frames.shape
    lib().synth_render_movers(_p(frames), N, H, W, _p(t), float(t_ref), _p(movers),
                              len(movers), float(fwhm))


def field_params(width, height, n_frames, t_ref, vx0, dvx, nvx, vy0, dvy, nvy, tau=5.0,
                 min_coverage=0):
    return dict(width=int(width), height=int(height), n_frames=int(n_frames),
                t_ref=float(t_ref), vx0=float(vx0), dvx=float(dvx), nvx=int(nvx),
                vy0=float(vy0), dvy=float(dvy), nvy=int(nvy), snr_threshold=float(tau),
                min_coverage=int(min_coverage))


def _place_movers(rng, M, W, H, t, t_ref, speed_fn, amp_fn, margin, integer=False,
                  vmax_int=10):
    dtmin, dtmax = float(np.min(t - t_ref)), float(np.max(t - t_ref))
    out = []
    tries = 0
    while len(out) < M:
        tries += 1
        if tries > 100000:
            raise RuntimeError("cannot place movers inside the field")
        if integer:
            vx, vy = (int(v) for v in rng.integers(-vmax_int, vmax_int + 1, size=2))
            x0, y0 = (int(v) for v in rng.integers(0, [W, H]))
        else:
            sp = speed_fn(rng)
            pa = rng.uniform(0.0, 2.0 * math.pi)
            vx, vy = sp * math.sin(pa), sp * math.cos(pa)
            x0, y0 = rng.uniform(0, W), rng.uniform(0, H)
        xs = [x0 + vx * dtmin, x0 + vx * dtmax]
        ys = [y0 + vy * dtmin, y0 + vy * dtmax]
        if min(xs) < margin or max(xs) > W - 1 - margin or min(ys) < margin or \
                max(ys) > H - 1 - margin:
            continue
        out.append([x0, y0, vx, vy, amp_fn(rng)])
    return np.array(out, np.float64)


def make_field(name, seed=None, **kw):
    """Returns dict(field=params, frames=f32 [N][H][W], times=f64 [N], truth=[M][5],
    unit=str, fwhm=float).  Keyword overrides: width, height, n_frames, n_movers,
    nv (grid size per axis, keeping the step), tau."""
    if seed is None:
        seed = BASE_SEED + {"tiny": 1, "mid": 2, "speculoos": 3, "batched": 4,
                            "refine": 5, "multinight": 6}.get(name, 0)
    rng = np.random.Generator(np.random.Philox(seed))
    fwhm = 3.0
    if name == "tiny":
        W = H = kw.get("width", 128)
        N = kw.get("n_frames", 16)
        t = np.arange(N, dtype=np.float64)
        t_ref = float(t[N // 2])
        nv = kw.get("nv", 21)
        f = field_params(W, H, N, t_ref, -(nv // 2), 1.0, nv, -(nv // 2), 1.0, nv,
                         kw.get("tau", 5.0))
        frames = noise(N, H, W, seed)
        truth = _place_movers(rng, kw.get("n_movers", 3), W, H, t, t_ref, None,
                              lambda r: 1.5, 2 * fwhm, integer=True, vmax_int=nv // 2)
        render_movers(frames, t, t_ref, truth, fwhm)
        return dict(field=f, frames=frames, times=t, truth=truth, unit="frame", fwhm=fwhm)
    if name == "mid":
        W = H = kw.get("width", 1024)
        N = kw.get("n_frames", 64)
        jitter = rng.uniform(-5.0, 5.0, size=N)
        t = (np.arange(N) * (7200.0 / max(N - 1, 1)) + jitter) / 3600.0
        t_ref = float(t[N // 2])
        nv = kw.get("nv", 161)
        f = field_params(W, H, N, t_ref, -0.5 * (nv // 2), 0.5, nv, -0.5 * (nv // 2), 0.5, nv,
                         kw.get("tau", 5.0))
        frames = noise(N, H, W, seed)
        lib().synth_add_smooth_residual(_p(frames), N, H, W, seed + 11, 2, 0.5)
        truth = _place_movers(rng, kw.get("n_movers", 20), W, H, t, t_ref,
                              lambda r: r.uniform(0.0, 40.0), lambda r: r.uniform(0.5, 3.0),
                              2 * fwhm)
        render_movers(frames, t, t_ref, truth, fwhm)
        nb = kw.get("n_blobs", 200)
        blobs = np.stack([rng.uniform(0, W, nb), rng.uniform(0, H, nb),
                          rng.uniform(3.0, 8.0, nb)], axis=1)
        lib().synth_mask_blobs(_p(frames), N, H, W, _p(np.ascontiguousarray(blobs)), nb)
        return dict(field=f, frames=frames, times=t, truth=truth, unit="h", fwhm=fwhm,
                    blobs=blobs)
    if name in ("speculoos", "refine"):
        W = H = kw.get("width", 2048)
        N = kw.get("n_frames", 256 if name == "speculoos" else 300)
        t = np.arange(N) * 50.0 / 3600.0
        t_ref = float(t[N // 2])
        nv = kw.get("nv", 801)
        f = field_params(W, H, N, t_ref, -0.25 * (nv // 2), 0.25, nv, -0.25 * (nv // 2), 0.25,
                         nv, kw.get("tau", 5.0))
        frames = noise(N, H, W, seed)
        hits = lib().synth_add_cosmics(_p(frames), N, H, W, seed + 7, 1e-5, 20.0, 200.0, None, 0)
        lo, hi = math.log(0.5), math.log(100.0)
        truth = _place_movers(rng, kw.get("n_movers", 100), W, H, t, t_ref,
                              lambda r: math.exp(r.uniform(lo, hi)),
                              lambda r: r.uniform(0.3, 3.0), 2 * fwhm)
        render_movers(frames, t, t_ref, truth, fwhm)
        return dict(field=f, frames=frames, times=t, truth=truth, unit="h", fwhm=fwhm,
                    n_cosmics=int(hits))
    if name == "multinight":
        W = H = kw.get("width", 1024)
        nights = kw.get("nights", 2)
        per = kw.get("n_frames", 128) // nights
        N = per * nights
        night = np.arange(per) * (2.0 / 60.0)            # 2 min cadence, hours
        t = np.concatenate([night + 24.0 * j for j in range(nights)])
        t_ref = float(0.5 * (t[0] + t[-1]))              # mid-baseline: |dt| <= baseline / 2
        vmax = kw.get("vmax", 5.0)
        base = float(t[-1] - t[0])
        dv = 1.0 / base                                   # 1 px over the whole baseline
        nv = kw.get("nv", 2 * int(math.floor(vmax / dv)) + 1)
        f = field_params(W, H, N, t_ref, -dv * (nv // 2), dv, nv, -dv * (nv // 2), dv, nv,
                         kw.get("tau", 5.0))
        frames = noise(N, H, W, seed)
        m = int(kw.get("n_movers", 10))
        truth = _place_movers(rng, m, W, H, t, t_ref, lambda r: r.uniform(0.0, vmax),
                              lambda r: r.uniform(0.3, 1.0), 2 * fwhm) if m else \
            np.zeros((0, 5))
        render_movers(frames, t, t_ref, truth, fwhm)
        return dict(field=f, frames=frames, times=t, truth=truth, unit="h", fwhm=fwhm)
    if name == "batched":
        j = kw.get("index", 0)
        rng, f, t, B = _batched_params(seed, j, kw)
        N, H, W, t_ref = f["n_frames"], f["height"], f["width"], f["t_ref"]
        frames = noise(N, H, W, seed + 1000 * j)
        M = int(kw.get("n_movers", rng.integers(10, 81)))
        truth = _place_movers(rng, M, W, H, t, t_ref, lambda r: r.uniform(0.0, 60.0),
                              lambda r: r.uniform(0.5, 3.0), 2 * fwhm)
        render_movers(frames, t, t_ref, truth, fwhm)
        return dict(field=f, frames=frames, times=t, truth=truth, unit="h", fwhm=fwhm)
    raise ValueError(f"unknown workload {name!r}")


def _batched_params(seed, j, kw):
    rng = np.random.Generator(np.random.Philox(seed + 1000 * j))
    N = int(kw.get("n_frames", rng.integers(40, 401)))
    W = H = int(kw.get("width", rng.choice([512, 1024, 2048])))
    B = float(kw.get("baseline", rng.uniform(1.0, 8.0)))
    t = np.linspace(0.0, B, N)
    t_ref = float(t[N // 2])
    dv = 1.0 / B
    nv = int(kw.get("nv", 2 * int(math.floor(60.0 * B)) + 1))
    f = field_params(W, H, N, t_ref, -dv * (nv // 2), dv, nv, -dv * (nv // 2), dv, nv,
                     kw.get("tau", 5.0))
    return rng, f, t, B


def batched_field(seed, index):
    """Parameters of field `index` of the batched workload (no frames drawn),
    identical to make_field("batched", seed=seed, index=index)["field"]."""
    return _batched_params(seed, index, {})[1]


def velocity_index(field, vx, vy):
    """Nearest grid index (a, b, k) of a velocity (input bookkeeping for recovery)."""
    a = int(round((vx - field["vx0"]) / field["dvx"]))
    b = int(round((vy - field["vy0"]) / field["dvy"]))
    a = min(max(a, 0), field["nvx"] - 1)
    b = min(max(b, 0), field["nvy"] - 1)
    return a, b, b * field["nvx"] + a
