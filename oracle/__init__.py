"""CPU oracle of the synthetic-tracking search (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is a ctypes wrapper around
``oracle.c`` (and ``refine_oracle.c``), a plain FP64 / FP32-sequential
restatement of the method of Burdanov, Hasler & de Wit (2023), Sec. 1 and
Sec. 2.1; it shares no code with the CUDA library.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OracleCand(C.Structure):
    _fields_ = [("x", C.c_int32), ("y", C.c_int32), ("k", C.c_int32), ("n_cov", C.c_int32),
                ("stack", C.c_double), ("snr", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.oracle_shift_tables.argtypes = [P, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int,
                                          C.c_int, P, P]
        L.oracle_sky_stats.argtypes = [P, C.c_int64, C.c_double, C.c_int, P, P, P, P]
        L.oracle_normalize.argtypes = [P, C.c_int, C.c_int64, C.c_double, C.c_int, C.c_float, P,
                                       P, P]
        L.oracle_round_bf16.argtypes = [P, C.c_int64, P]
        grid = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_double, C.c_double, C.c_int]
        L.oracle_stack_planes.argtypes = [P, C.c_int, C.c_int, C.c_int, P] + grid + [
            C.c_int, C.c_int, P, C.c_int, P, P]
        L.oracle_stack_points.argtypes = [P, C.c_int, C.c_int, C.c_int, P] + grid + [
            C.c_int, C.c_int, P, C.c_int64, P, P]
        L.oracle_search.argtypes = [P, C.c_int, C.c_int, C.c_int, P] + grid + [
            C.c_int, C.c_int, C.c_float, C.c_int, C.c_int32, C.c_int32, P, C.c_int64]
        L.oracle_search.restype = C.c_int64
        L.oracle_num_threads.restype = C.c_int
        L.oracle_set_num_threads.argtypes = [C.c_int]
        L.oracle_set_num_threads.restype = None
        L.oracle_refine_eval.argtypes = [P, C.c_int, C.c_int, C.c_int, P, C.c_double, P, P,
                                         C.c_int64, C.c_double, P, P, P]
        L.oracle_refine_gn_matrix.argtypes = [C.c_int, P, C.c_double, P, P, C.c_int64,
                                              C.c_double, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_num_threads(n: int) -> None:
    lib().oracle_set_num_threads(int(n))


def shift_tables(t, t_ref, v0, dv, nv, mode="nearest"):
    """Shift table [N][nv] (int32) and fractions [N][nv] (FP64)."""
    t = _f64(t)
    s = np.zeros((t.size, nv), np.int32)
    f = np.zeros((t.size, nv), np.float64)
    lib().oracle_shift_tables(_p(t), t.size, t_ref, v0, dv, nv, 0 if mode == "nearest" else 1,
                              _p(s), _p(f))
    return s, f


def sky_stats(frame, kappa=3.0, max_iter=5):
    x = _f32(frame).ravel()
    mu = C.c_double()
    sd = C.c_double()
    kept = C.c_int64()
    it = C.c_int()
    lib().oracle_sky_stats(_p(x), x.size, kappa, max_iter, C.byref(mu), C.byref(sd),
                           C.byref(kept), C.byref(it))
    return mu.value, sd.value, kept.value, it.value


def normalize(raw, kappa=3.0, max_iter=5, cr_clip=0.0):
    raw = _f32(raw)
    N = raw.shape[0]
    npix = raw[0].size
    out = np.empty_like(raw)
    mu = np.zeros(N)
    sd = np.zeros(N)
    lib().oracle_normalize(_p(raw), N, npix, kappa, max_iter, cr_clip, _p(out), _p(mu), _p(sd))
    return out, mu, sd


def round_bf16(x):
    x = _f32(x)
    out = np.empty_like(x)
    lib().oracle_round_bf16(_p(x), x.size, _p(out))
    return out


def _grid(field):
    return (float(field["t_ref"]), float(field["vx0"]), float(field["dvx"]), int(field["nvx"]),
            float(field["vy0"]), float(field["dvy"]), int(field["nvy"]))


def stack_planes(frames, t, field, ks, mode="nearest", prec="fp64"):
    """S [len(ks)][H][W] (float64 holding FP32 values in 'fp32' mode) and n_cov."""
    frames = _f32(frames)
    t = _f64(t)
    N, H, W = frames.shape
    ks = np.ascontiguousarray(ks, dtype=np.int32)
    S = np.zeros((ks.size, H, W), np.float64)
    Cv = np.zeros((ks.size, H, W), np.int32)
    lib().oracle_stack_planes(_p(frames), N, H, W, _p(t), *_grid(field),
                              0 if mode == "nearest" else 1, 0 if prec == "fp64" else 1,
                              _p(ks), ks.size, _p(S), _p(Cv))
    return S, Cv


def stack_points(frames, t, field, xyk, mode="nearest", prec="fp64"):
    frames = _f32(frames)
    t = _f64(t)
    N, H, W = frames.shape
    xyk = np.ascontiguousarray(xyk, dtype=np.int32).reshape(-1, 3)
    S = np.zeros(len(xyk), np.float64)
    Cv = np.zeros(len(xyk), np.int32)
    lib().oracle_stack_points(_p(frames), N, H, W, _p(t), *_grid(field),
                              0 if mode == "nearest" else 1, 0 if prec == "fp64" else 1,
                              _p(xyk), len(xyk), _p(S), _p(Cv))
    return S, Cv


def candidates_at(frames, t, field, xyk, mode="nearest", prec="fp32"):
    """The detection rule of Sec. 2.1 evaluated point by point, for fields too
    large to search whole: for each (x, y, k) row of xyk, whether it is a
    candidate (coverage n_cov >= n_min, S >= fl32(tau sqrt(n_cov)), and a
    local maximum of S_k over the in-frame neighbours with n_cov >= n_min:
    strictly above earlier neighbours in raster order, at least equal to
    later ones), with its S, n_cov and S/N.  The same rule as ``search``,
    with S and n_cov of the point and its 8 neighbours from ``stack_points``.
    Returns (is_cand bool [n], S float64 [n], n_cov int32 [n], snr float64 [n])."""
    xyk = np.ascontiguousarray(xyk, dtype=np.int64).reshape(-1, 3)
    W, H, N = int(field["width"]), int(field["height"]), int(field["n_frames"])
    nmin = int(field.get("min_coverage", 0)) or (N + 1) // 2
    tau = np.float32(field["snr_threshold"])
    n = len(xyk)
    offs = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]   # raster order; centre j = 4
    pts = np.repeat(xyk, 9, axis=0)
    pts[:, 0] += np.tile([dx for dx, _ in offs], n)
    pts[:, 1] += np.tile([dy for _, dy in offs], n)
    inside = (pts[:, 0] >= 0) & (pts[:, 0] < W) & (pts[:, 1] >= 0) & (pts[:, 1] < H)
    S = np.zeros(len(pts))
    Cv = np.zeros(len(pts), np.int32)
    if inside.any():
        S[inside], Cv[inside] = stack_points(frames, t, field, pts[inside], mode, prec)
    S, Cv, inside = S.reshape(n, 9), Cv.reshape(n, 9), inside.reshape(n, 9)
    s, c = S[:, 4], Cv[:, 4]
    th = (np.float64(tau) * np.sqrt(c.astype(np.float64))).astype(np.float32)
    if prec == "fp32":
        above = s.astype(np.float32) >= th
        rsq = np.where(c > 0, 1.0 / np.sqrt(np.maximum(c, 1).astype(np.float64)), 0.0)
        snr = (s.astype(np.float32) * rsq.astype(np.float32)).astype(np.float64)
    else:
        above = s >= th.astype(np.float64)
        snr = s / np.sqrt(np.maximum(c, 1).astype(np.float64))
    ok = inside[:, 4] & (c >= nmin) & above
    for j in range(9):
        if j == 4:
            continue
        live = inside[:, j] & (Cv[:, j] >= nmin)
        beats = s > S[:, j] if j < 4 else s >= S[:, j]
        ok &= beats | ~live
    return ok, s, c, snr


def search(frames, t, field, mode="nearest", prec="fp32", k_begin=0, k_end=None, cap=None):
    """Sorted candidates as a structured numpy array (x, y, k, n_cov, stack, snr)."""
    frames = _f32(frames)
    t = _f64(t)
    N, H, W = frames.shape
    nk = int(field["nvx"]) * int(field["nvy"])
    if k_end is None:
        k_end = nk
    args = (_p(frames), N, H, W, _p(t), *_grid(field), 0 if mode == "nearest" else 1,
            0 if prec == "fp64" else 1, float(field["snr_threshold"]),
            int(field.get("min_coverage", 0)), int(k_begin), int(k_end))
    L = lib()
    explicit = cap is not None
    cap = cap if explicit else 1 << 18
    buf = (OracleCand * max(cap, 1))()
    n = L.oracle_search(*args, C.cast(buf, C.c_void_p), cap)
    if n < 0:
        raise MemoryError("oracle_search allocation failed")
    if n > cap and not explicit:
        cap = n
        buf = (OracleCand * cap)()
        n = L.oracle_search(*args, C.cast(buf, C.c_void_p), cap)
    dt = np.dtype([("x", np.int32), ("y", np.int32), ("k", np.int32), ("n_cov", np.int32),
                   ("stack", np.float64), ("snr", np.float64)])
    arr = np.frombuffer(bytearray(buf), dtype=dt, count=min(n, cap)).copy()
    return arr


def refine_eval(frames, t, t_ref, theta, centre, fwhm=3.0, grad=True):
    """FP64 refinement objective: J [n], SNR [n] and dJ/dtheta [n][5]
    (theta rows: vx, vy, x0, y0, F; centre rows: integer cutout centre)."""
    frames = _f32(frames)
    t = _f64(t)
    N, H, W = frames.shape
    th = _f64(theta).reshape(-1, 5)
    ce = np.ascontiguousarray(centre, np.int32).reshape(-1, 2)
    n = len(th)
    J = np.zeros(n)
    snr = np.zeros(n)
    g = np.zeros((n, 5)) if grad else None
    lib().oracle_refine_eval(_p(frames), N, H, W, _p(t), float(t_ref), _p(th), _p(ce), n,
                             float(fwhm), _p(J), _p(snr), _p(g) if grad else None)
    return J, snr, g


def refine_gn_matrix(t, t_ref, theta, centre, fwhm=3.0):
    """Gauss-Newton curvature J^T J [n][5][5] of the refinement objective at
    theta (order vx, vy, x0, y0, F; refine_oracle.c states the entries)."""
    t = _f64(t)
    th = _f64(theta).reshape(-1, 5)
    ce = np.ascontiguousarray(centre, np.int32).reshape(-1, 2)
    n = len(th)
    H = np.zeros((n, 5, 5))
    lib().oracle_refine_gn_matrix(len(t), _p(t), float(t_ref), _p(th), _p(ce), n, float(fwhm),
                                  _p(H))
    return H


def refine_gn_step(frames, t, t_ref, theta, centre, fwhm=3.0, damping=0.0):
    """One Gauss-Newton step of the refinement with the flux profiled out, in
    the order the library's refinement takes a step: F is first set to its
    optimum <g,S>/(N <g,g>) at the current motion and position, then
    (vx, vy, x0, y0) move by the solution of
        (Hs + damping diag(Hs)) delta = dJ/d(vx, vy, x0, y0),
    Hs the Schur complement of the F entry in J^T J (the curvature of J with
    F at its optimum).  Returns the new theta rows."""
    th = _f64(theta).reshape(-1, 5).copy()
    N = len(t)
    H0 = refine_gn_matrix(t, t_ref, th, centre, fwhm)
    J, snr, _ = refine_eval(frames, t, t_ref, th, centre, fwhm, grad=False)
    gg = H0[:, 4, 4] / N
    th[:, 4] = snr * np.sqrt(N * gg) / (N * gg)          # <g,S> / (N <g,g>)
    _, _, g = refine_eval(frames, t, t_ref, th, centre, fwhm)
    H = refine_gn_matrix(t, t_ref, th, centre, fwhm)
    Hs = H[:, :4, :4] - H[:, :4, 4:5] * H[:, 4:5, :4] / H[:, 4:5, 4:5]
    A = Hs + damping * Hs * np.eye(4)[None]
    delta = np.linalg.solve(A, g[:, :4, None])[:, :, 0]
    th[:, :4] += delta
    return th
