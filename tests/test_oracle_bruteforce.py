"""Brute force on tiny inputs (CPU only): an independent numpy statement of
the stack and candidate rule, exhaustive over every velocity and pixel,
checked against the C oracle.  Sec. 1 / Sec. 2.1 of Burdanov, Hasler &
de Wit (2023); the readings are those of oracle/oracle.c's header.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def brute_stack(fr, t, f, mode):
    N, H, W = fr.shape
    out = np.zeros((f["nvy"], f["nvx"], H, W))
    cov = np.zeros((f["nvy"], f["nvx"], H, W), np.int64)
    pad = np.zeros((N, H + 2, W + 2))
    pad[:, :H, :W] = fr  # taps beyond the frame read 0 (extra zero row/column)
    for b in range(f["nvy"]):
        for a in range(f["nvx"]):
            vx = f["vx0"] + a * f["dvx"]
            vy = f["vy0"] + b * f["dvy"]
            for i in range(N):
                dt = t[i] - f["t_ref"]
                for y in range(H):
                    for x in range(W):
                        px, py = x + vx * dt, y + vy * dt
                        if mode == "nearest":
                            u, v = math.floor(px + 0.5), math.floor(py + 0.5)
                            if 0 <= u < W and 0 <= v < H:
                                out[b, a, y, x] += fr[i, v, u]
                                cov[b, a, y, x] += 1
                        else:
                            u, v = math.floor(px), math.floor(py)
                            gx, gy = px - u, py - v
                            val = 0.0
                            for (du, dv, w) in ((0, 0, (1 - gx) * (1 - gy)), (1, 0, gx * (1 - gy)),
                                                (0, 1, (1 - gx) * gy), (1, 1, gx * gy)):
                                uu, vv = u + du, v + dv
                                if 0 <= uu < W and 0 <= vv < H:
                                    val += w * pad[i, vv, uu]
                            out[b, a, y, x] += val
                            if 0 <= px <= W - 1 and 0 <= py <= H - 1:
                                cov[b, a, y, x] += 1
    return out.reshape(-1, H, W), cov.reshape(-1, H, W)


def brute_candidates(S, Cv, tau, nmin):
    K, H, W = S.shape
    res = []
    for k in range(K):
        for y in range(H):
            for x in range(W):
                c = Cv[k, y, x]
                if c < nmin or not S[k, y, x] >= np.float32(tau * math.sqrt(c)):
                    continue
                ok = True
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        if (dx, dy) == (0, 0):
                            continue
                        qx, qy = x + dx, y + dy
                        if not (0 <= qx < W and 0 <= qy < H) or Cv[k, qy, qx] < nmin:
                            continue
                        if (dy, dx) < (0, 0):
                            ok &= S[k, y, x] > S[k, qy, qx]
                        else:
                            ok &= S[k, y, x] >= S[k, qy, qx]
                if ok:
                    res.append((x, y, k, c))
    return res


@pytest.mark.parametrize("mode", ["nearest", "bilinear"])
@pytest.mark.parametrize("seed", [1, 2])
def test_bruteforce_planes_and_candidates(mode, seed):
    rng = np.random.default_rng(seed)
    N, H, W = 5, 9, 11
    fr = synth.noise(N, H, W, seed=100 + seed)
    fr[rng.integers(0, N), 4, 5] += 6.0
    t = np.sort(rng.uniform(0, 4, N))
    f = synth.field_params(W, H, N, float(t[2]), -1.1, 0.7, 4, 0.6, -0.55, 3, tau=1.5)
    S, Cv = oracle.stack_planes(fr, t, f, np.arange(12), mode=mode)
    Sb, Cb = brute_stack(fr.astype(np.float64), t, f, mode)
    assert np.array_equal(Cv, Cb)
    assert np.max(np.abs(S - Sb)) < 1e-12
    nmin = (N + 1) // 2
    c = oracle.search(fr, t, f, mode=mode, prec="fp64")
    got = [(int(r["x"]), int(r["y"]), int(r["k"]), int(r["n_cov"])) for r in c]
    assert got == brute_candidates(Sb, Cb, 1.5, nmin)
