"""Pins of the CPU oracle to facts outside itself (CPU only).

Each test states the fact it checks: a closed form, an invariant of the
shift-and-stack of Burdanov, Hasler & de Wit (2023) Sec. 1 / Sec. 2.1, a
special case that reduces to a library routine, statistics of pure noise, or
a hand-derived fixture in tests/golden/.  Together they catch a wrong shift
sign, swapped axes, a wrong rounding rule, a dropped or mis-weighted bilinear
tap, a wrong threshold comparison or tie rule, and a wrong coverage count.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def grid_field(W, H, N, t_ref, vx0, dvx, nvx, vy0, dvy, nvy, tau=5.0, nmin=0):
    return synth.field_params(W, H, N, t_ref, vx0, dvx, nvx, vy0, dvy, nvy, tau, nmin)


# --------------------------------------------------------------- a1 shifts

def test_shift_nearest_hand_cases():
    # v in {-1,-0.5,0,0.5,1}; dt in {-1, 0, 2}.  floor(v*dt + 0.5) by hand.
    s, f = oracle.shift_tables([0.0, 1.0, 3.0], 1.0, -1.0, 0.5, 5, "nearest")
    assert s.tolist() == [[1, 1, 0, 0, -1], [0, 0, 0, 0, 0], [-2, -1, 0, 1, 2]]
    assert np.all(f == 0)


def test_shift_bilinear_hand_cases():
    # floor(v*dt) and the fraction, by hand: dt=-1 -> s = 1, .5, 0, -.5, -1
    s, f = oracle.shift_tables([0.0, 1.0, 3.0], 1.0, -1.0, 0.5, 5, "bilinear")
    assert s[0].tolist() == [1, 0, 0, -1, -1]
    assert f[0].tolist() == [0.0, 0.5, 0.0, 0.5, 0.0]
    assert s[2].tolist() == [-2, -1, 0, 1, 2]
    # fraction of 0.3*1.7: 0.51 - floor -> in [0, 1)
    s2, f2 = oracle.shift_tables([1.7], 0.0, 0.3, 1.0, 1, "bilinear")
    assert s2[0, 0] == 0 and abs(f2[0, 0] - 0.51) < 1e-15


# ------------------------------------------------------- a2 sky statistics

def test_sky_stats_clipped_closed_form():
    # 10000 pixels at c-1 / c+1 (mean c, population std 1), two outliers at
    # c+100 and two NaNs.  First pass: std ~1.73, the outliers sit ~57 std out
    # and are clipped; second pass: mean c and std 1 exactly; the set is then
    # unchanged, so two passes.
    c = 37.0
    x = np.full(10004, c, np.float32)
    x[:5000] = c - 1
    x[5000:10000] = c + 1
    x[10000:10002] = c + 100
    x[10002:] = np.nan
    mu, sd, kept, it = oracle.sky_stats(x)
    assert mu == c and sd == 1.0 and kept == 10000 and it == 2


def test_sky_stats_gaussian_matches_clipped_normal():
    # Clipping a unit normal at 3 sigma leaves std sqrt(1 - 6 phi(3)/(2 Phi(3)-1))
    # at the fixed point; with 4M samples the estimate is within a few 1e-3.
    x = synth.noise(1, 2048, 2048, seed=99)[0] * 2.5 + 10.0
    mu, sd, kept, it = oracle.sky_stats(x)
    assert abs(mu - 10.0) < 5e-3
    # iterate the truncation to its fixed point analytically (standard normal)
    from math import erf, exp, pi, sqrt
    s = 1.0
    for _ in range(5):
        a = 3.0 * s
        phi = exp(-a * a / 2) / sqrt(2 * pi)
        P = erf(a / sqrt(2))
        s = sqrt(1 - 2 * a * phi / P)
    assert abs(sd / 2.5 - s) < 5e-3
    assert 1 <= it <= 5


def test_normalize_closed_form_nan_and_clip():
    N, H, W = 3, 4, 6
    raw = np.empty((N, H, W), np.float32)
    pat = np.where((np.arange(H * W) % 2) == 0, -1.0, 1.0).reshape(H, W)
    for i in range(N):
        raw[i] = 100.0 * (i + 1) + 4.0 * pat   # mean 100(i+1), std 4
    raw[1, 0, 0] = np.nan
    out, mu, sd = oracle.normalize(raw)
    assert out[1, 0, 0] == 0.0
    good = np.isfinite(raw)
    # frame 0, 2: exactly +-1 after normalisation
    assert np.array_equal(out[0], pat.astype(np.float32))
    assert np.array_equal(out[2], pat.astype(np.float32))
    assert mu[0] == 100.0 and sd[0] == 4.0
    # cosmic-ray clip zeroes |I| > clip
    raw2 = raw.copy()
    raw2[0, 2, 2] = 1e6
    out2, _, _ = oracle.normalize(raw2, cr_clip=10.0)
    assert out2[0, 2, 2] == 0.0
    assert good.sum() == N * H * W - 1


def test_normalize_degenerate_frames():
    # no finite pixel: no statistics (mu = sigma = 0); a constant frame: no
    # scatter (sigma = 0); both map to zeros, the frame between is untouched
    raw = np.empty((3, 5, 8), np.float32)
    raw[0] = np.nan
    raw[1] = np.where((np.arange(40) % 2) == 0, 3.0, 5.0).reshape(5, 8)  # mean 4, std 1
    raw[2] = 7.25
    out, mu, sd = oracle.normalize(raw)
    assert mu[0] == 0.0 and sd[0] == 0.0 and np.all(out[0] == 0.0)
    assert mu[2] == 7.25 and sd[2] == 0.0 and np.all(out[2] == 0.0)
    assert mu[1] == 4.0 and sd[1] == 1.0
    assert np.array_equal(out[1], raw[1] - 4.0)


# ------------------------------------------------------ a3 nearest stacking

@pytest.fixture(scope="module")
def small_noise():
    N, H, W = 12, 40, 56
    fr = synth.noise(N, H, W, seed=7)
    t = np.array([0.0, 0.9, 2.1, 3.0, 4.2, 4.9, 6.1, 7.0, 8.3, 8.8, 10.1, 11.0])
    return fr, t


def test_zero_velocity_is_frame_sum(small_noise):
    fr, t = small_noise
    N, H, W = fr.shape
    f = grid_field(W, H, N, 5.0, -1.0, 0.5, 5, -1.0, 0.5, 5)
    k0 = 2 * 5 + 2  # a = b = 2 -> v = 0
    S, Cv = oracle.stack_planes(fr, t, f, [k0], prec="fp64")
    assert np.all(Cv == N)
    ref = fr.astype(np.float64).sum(axis=0)
    assert np.max(np.abs(S[0] - ref)) < 1e-12
    # FP32 sequential mode == numpy's sequential float32 running sum
    S32, _ = oracle.stack_planes(fr, t, f, [k0], prec="fp32")
    seq = np.cumsum(fr, axis=0, dtype=np.float32)[-1]
    assert np.array_equal(S32[0].astype(np.float32), seq)


def test_noiseless_injection_recovers_truth():
    # Non-square frame, integer times and velocity with vx != vy, both != 0.
    N, H, W = 10, 48, 64
    t = np.arange(N, dtype=np.float64)
    t_ref = 4.0
    x0, y0, vx, vy, A = 30, 20, 2, -1, 1.0
    fr = np.zeros((N, H, W), np.float32)
    synth.render_movers(fr, t, t_ref, [[x0, y0, vx, vy, A]], fwhm=3.0)
    F = float(fr[int(t_ref)].astype(np.float64).sum())  # discrete flux of one frame
    f = grid_field(W, H, N, t_ref, -3, 1, 7, -3, 1, 7, tau=1.0)
    ks = np.arange(49)
    S, Cv = oracle.stack_planes(fr, t, f, ks, prec="fp64")
    k_true = (vy + 3) * 7 + (vx + 3)
    kk, yy, xx = np.unravel_index(np.argmax(S), S.shape)
    assert (kk, yy, xx) == (k_true, y0, x0)
    assert abs(S[k_true, y0, x0] - N * A) < 1e-5
    ap = S[k_true, y0 - 6:y0 + 7, x0 - 6:x0 + 7].sum()
    assert abs(ap - N * F) < 1e-4
    c = oracle.search(fr, t, f, prec="fp32")
    best = c[np.argmax(c["stack"])]
    assert (best["x"], best["y"], best["k"]) == (x0, y0, k_true)


def test_linearity(small_noise):
    fr, t = small_noise
    N, H, W = fr.shape
    g = synth.noise(N, H, W, seed=8)
    f = grid_field(W, H, N, 5.0, -1.3, 0.7, 4, 0.4, -0.6, 3)
    ks = [0, 5, 11]
    a, b = 1.75, -0.5
    Sa, _ = oracle.stack_planes(fr, t, f, ks)
    Sb, _ = oracle.stack_planes(g, t, f, ks)
    X = (a * fr + b * g).astype(np.float32)
    # X carries the FP32 rounding of the combination; its stack is bounded by N max|err|
    err = np.max(np.abs(X.astype(np.float64) - (a * fr.astype(np.float64) + b * g)))
    Sab, _ = oracle.stack_planes(X, t, f, ks)
    assert np.max(np.abs(Sab - (a * Sa + b * Sb))) <= N * err + 1e-12
    # powers of two are exact in FP32
    S1, _ = oracle.stack_planes(fr, t, f, ks, prec="fp32")
    S2, _ = oracle.stack_planes(4.0 * fr, t, f, ks, prec="fp32")
    assert np.array_equal(S2, 4.0 * S1)


def test_time_reversal(small_noise):
    # S_v(t, t_ref) == S_{-v}(-t, -t_ref): same samples in the same order.
    fr, t = small_noise
    N, H, W = fr.shape
    f = grid_field(W, H, N, 5.0, -1.2, 0.6, 5, -0.9, 0.45, 5)
    fr_ = grid_field(W, H, N, -5.0, -1.2, 0.6, 5, -0.9, 0.45, 5)
    for mode in ("nearest", "bilinear"):
        for (a, b) in [(0, 1), (4, 3), (1, 4)]:
            S, C1 = oracle.stack_planes(fr, t, f, [b * 5 + a], mode=mode, prec="fp32")
            Sr, C2 = oracle.stack_planes(fr, -t, fr_, [(4 - b) * 5 + (4 - a)], mode=mode,
                                         prec="fp32")
            if mode == "nearest":
                assert np.array_equal(S, Sr) and np.array_equal(C1, C2)
            else:
                assert np.max(np.abs(S - Sr)) < 1e-5 and np.array_equal(C1, C2)


def test_translation_equivariance(small_noise):
    fr, t = small_noise
    N, H, W = fr.shape
    f = grid_field(W, H, N, 5.0, -1.0, 0.5, 5, -1.0, 0.5, 5)
    dx, dy = 3, -2
    moved = np.zeros_like(fr)
    moved[:, max(dy, 0):H + min(dy, 0), max(dx, 0):W + min(dx, 0)] = \
        fr[:, max(-dy, 0):H - max(dy, 0), max(-dx, 0):W - max(dx, 0)]
    S, _ = oracle.stack_planes(fr, t, f, [7], prec="fp32")
    Sm, _ = oracle.stack_planes(moved, t, f, [7], prec="fp32")
    # interior: far from edges by more than max |shift| (<= 1 * 6) + |d|
    m = 12
    assert np.array_equal(Sm[0, m + dy:H - m + dy, m + dx:W - m + dx], S[0, m:H - m, m:W - m])


def test_pure_noise_stack_has_sigma_sqrt_n():
    N, H, W = 64, 96, 96
    fr = synth.noise(N, H, W, seed=11)
    t = np.arange(N) / 8.0
    f = grid_field(W, H, N, 4.0, -2.0, 1.0, 5, -2.0, 1.0, 5)
    S, Cv = oracle.stack_planes(fr, t, f, [3, 12, 21])
    inner = S[:, 16:-16, 16:-16]
    assert np.all(Cv[:, 16:-16, 16:-16] == N)
    n = inner[0].size
    for p in inner:
        # sample std of n iid N(0, N): relative s.e. 1/sqrt(2n); 5 sigma band
        assert abs(p.std() / math.sqrt(N) - 1) < 5 / math.sqrt(2 * n)
        assert abs(p.mean()) < 5 * math.sqrt(N / n)


# ---------------------------------------------------- a4 bilinear stacking

def test_bilinear_equals_nearest_for_integer_shifts(small_noise):
    fr, _ = small_noise
    N, H, W = fr.shape
    t = np.arange(N, dtype=np.float64)
    f = grid_field(W, H, N, 6.0, -2.0, 1.0, 5, -1.0, 1.0, 3)
    ks = list(range(15))
    Sn, Cn = oracle.stack_planes(fr, t, f, ks, mode="nearest")
    Sb, Cb = oracle.stack_planes(fr, t, f, ks, mode="bilinear")
    assert np.array_equal(Cn, Cb)
    assert np.max(np.abs(Sn - Sb)) < 1e-12


def test_bilinear_linear_ramp_closed_form():
    # Bilinear interpolation reproduces a linear function exactly:
    # S = sum_i [alpha (x + vx dt_i) + beta (y + vy dt_i) + gamma].
    N, H, W = 9, 30, 40
    t = np.array([0.0, 0.37, 1.1, 1.5, 2.25, 2.9, 3.3, 4.05, 4.6])
    al, be, ga = 0.25, -0.125, 2.0
    yy, xx = np.mgrid[0:H, 0:W]
    fr = np.broadcast_to((al * xx + be * yy + ga).astype(np.float32), (N, H, W)).copy()
    f = grid_field(W, H, N, 2.25, -1.3, 0.55, 6, 0.7, -0.45, 4)
    ks = np.arange(24)
    S, Cv = oracle.stack_planes(fr, t, f, ks, mode="bilinear")
    dt = t - 2.25
    m = 8
    for q, k in enumerate(ks):
        a, b = k % 6, k // 6
        vx, vy = -1.3 + a * 0.55, 0.7 + b * -0.45
        ref = (al * (xx[None] + vx * dt[:, None, None]) + be * (yy[None] + vy * dt[:, None, None])
               + ga).sum(axis=0)
        assert np.all(Cv[q, m:-m, m:-m] == N)
        assert np.max(np.abs(S[q, m:-m, m:-m] - ref[m:-m, m:-m])) < 1e-9


def test_bilinear_constant_frames():
    N, H, W = 7, 20, 20
    t = np.linspace(0, 3.1, N)
    fr = np.full((N, H, W), 1.5, np.float32)
    f = grid_field(W, H, N, 1.3, -0.77, 0.31, 6, 0.2, 0.43, 3)
    S, Cv = oracle.stack_planes(fr, t, f, np.arange(18), mode="bilinear")
    assert np.max(np.abs(S[:, 5:-5, 5:-5] - 1.5 * N)) < 1e-12
    assert np.all(Cv[:, 5:-5, 5:-5] == N)


def test_bilinear_noise_variance_matches_weights():
    # For iid unit-variance frames the interior variance of a bilinear stack
    # is sum_i ((1-fx)^2 + fx^2)((1-fy)^2 + fy^2): pins the tap weights.
    N, H, W = 40, 128, 128
    fr = synth.noise(N, H, W, seed=21)
    t = np.arange(N) * 0.173
    f = grid_field(W, H, N, t[N // 2], 0.9, 0.37, 3, -1.1, 0.29, 3)
    ks = [4, 8]
    S, _ = oracle.stack_planes(fr, t, f, ks, mode="bilinear")
    for q, k in enumerate(ks):
        a, b = k % 3, k // 3
        vx, vy = 0.9 + a * 0.37, -1.1 + b * 0.29
        dt = t - t[N // 2]
        fx = vx * dt - np.floor(vx * dt)
        fy = vy * dt - np.floor(vy * dt)
        var = np.sum(((1 - fx) ** 2 + fx ** 2) * ((1 - fy) ** 2 + fy ** 2))
        p = S[q, 20:-20, 20:-20]
        # neighbouring outputs share taps; use a sparse lattice of independent ones
        pts = p[::3, ::3]
        n = pts.size
        assert abs(pts.var() / var - 1) < 5 * math.sqrt(2.0 / n)
        # and the nominal sqrt(N) would be far off for these fractions
        assert var < 0.9 * N


def test_bilinear_coverage_rule_edge():
    # in-bounds iff 0 <= x + s <= W-1: with vx = 0.5, dt = 1 the last pixel
    # x = W-1 samples W-0.5 (outside) and x = W-2 samples W-1.5 (inside).
    N, H, W = 2, 5, 6
    t = np.array([0.0, 1.0])
    fr = np.ones((N, H, W), np.float32)
    f = grid_field(W, H, N, 0.0, 0.5, 1.0, 1, 0.0, 1.0, 1)
    S, Cv = oracle.stack_planes(fr, t, f, [0], mode="bilinear")
    assert Cv[0, 2, W - 1] == 1 and Cv[0, 2, W - 2] == 2
    # the outside sample still interpolates its inside tap with weight 1/2
    assert S[0, 2, W - 1] == 1.5 and S[0, 2, W - 2] == 2.0


# ------------------------------------------------- a5/a6 candidate fixtures

def _golden_cases():
    with open(os.path.join(GOLDEN, "candidate_rules.json")) as fh:
        return json.load(fh)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_candidate_rule_fixtures(case):
    N, H, W = case["N"], case["H"], case["W"]
    fr = np.zeros((N, H, W), np.float32)
    for (i, x, y, v) in case["points"]:
        fr[i, y, x] = v
    vx0, dvx, nvx, vy0, dvy, nvy = case["grid"]
    f = grid_field(W, H, N, case["t_ref"], vx0, dvx, int(nvx), vy0, dvy, int(nvy),
                   case["tau"], case["min_coverage"])
    for prec in ("fp32", "fp64"):
        c = oracle.search(fr, np.array(case["times"], np.float64), f, prec=prec)
        got = [[int(r["x"]), int(r["y"]), int(r["k"]), int(r["n_cov"]), float(r["stack"])]
               for r in c]
        assert got == [e[:5] for e in case["expected"]], prec
        if prec == "fp32":
            assert [float(np.float32(r["snr"])) for r in c] == [e[5] for e in case["expected"]]


def test_candidates_sorted_by_k_then_raster():
    d = synth.make_field("tiny", width=64, n_frames=12, n_movers=3, tau=4.0)
    c = oracle.search(d["frames"], d["times"], d["field"], prec="fp32")
    key = c["k"].astype(np.int64) << 32 | c["y"].astype(np.int64) << 16 | c["x"]
    assert len(c) > 3 and np.all(np.diff(key) > 0)


# ------------------------------------------------- a7 BF16 storage rounding

def _f32_bits(u):
    return np.array(u, dtype=np.uint32).view(np.float32)


def _bits(x):
    return np.asarray(x, np.float32).view(np.uint32)


def test_round_bf16_hand_cases():
    # A BF16 value is an FP32 value whose low 16 bits are zero; storing an
    # FP32 in BF16 rounds to the nearest such value, ties to the one whose
    # bit 16 is zero (IEEE round to nearest even).
    cases = [
        (0x3F808000, 0x3F800000),  # tie, kept bit 16 even -> round down
        (0x3F818000, 0x3F820000),  # tie, bit 16 odd -> round up to even
        (0x3F807FFF, 0x3F800000),  # just below a tie -> down
        (0x3F808001, 0x3F810000),  # just above a tie -> up
        (0x3F81FFFF, 0x3F820000),  # carries into the next bf16 value
        (0xBF808000, 0xBF800000),  # negative tie, even -> toward zero
        (0xBF818000, 0xBF820000),  # negative tie, odd -> away from zero
        (0x00000000, 0x00000000),  # +0
        (0x80000000, 0x80000000),  # -0 keeps its sign
        (0x00008000, 0x00000000),  # subnormal tie, even -> 0
        (0x00018000, 0x00020000),  # subnormal tie, odd -> up
        (0x00007FFF, 0x00000000),  # tiny subnormal -> +0
        (0x807FFFFF, 0x80800000),  # largest negative subnormal -> -min normal
        (0x7F7FFFFF, 0x7F800000),  # largest finite rounds to +inf
        (0x7F7F7FFF, 0x7F7F0000),  # largest finite bf16 stays
        (0xFF7F8000, 0xFF800000),  # tie at the top, odd -> -inf
        (0x7F800000, 0x7F800000),  # +inf
        (0xFF800000, 0xFF800000),  # -inf
    ]
    x = _f32_bits([c[0] for c in cases])
    got = _bits(oracle.round_bf16(x))
    assert [hex(g) for g in got] == [hex(c[1]) for c in cases]


def test_round_bf16_nan_stays_nan():
    # a NaN whose payload sits only in the low 16 bits must not become inf
    x = _f32_bits([0x7F800001, 0xFF800001, 0x7FC00000, 0x7F80FFFF])
    got = oracle.round_bf16(x)
    assert np.all(np.isnan(got))
    assert np.all(_bits(got) & 0xFFFF == 0)


def _round_bf16_by_definition(x):
    # nearest of the two neighbouring BF16 values (exact differences in
    # FP64); ties to the one with bit 16 clear; inf beyond the largest
    u = _bits(x).astype(np.uint64)
    lo = (u & 0xFFFF0000).astype(np.uint32)
    hi = (lo.astype(np.uint64) + 0x10000).astype(np.uint32)
    xl = lo.view(np.float32).astype(np.float64)
    xh = hi.view(np.float32).astype(np.float64)
    # past the largest BF16 the next value up is 2^128 (unbounded exponent),
    # stored as inf: IEEE rounding overflows from the midpoint on
    xh = np.where(np.isinf(xh), np.copysign(2.0 ** 128, xh), xh)
    xv = np.asarray(x, np.float32).astype(np.float64)
    dl, dh = np.abs(xv - xl), np.abs(xh - xv)
    even_lo = ((lo >> 16) & 1) == 0
    pick_lo = (dl < dh) | ((dl == dh) & even_lo)
    return np.where(pick_lo, lo, hi).astype(np.uint32)  # hi of 2^128 is the inf pattern


def test_round_bf16_dense_sweep_against_definition_and_torch():
    # every 257th bit pattern (all exponents, signs and low-bit phases) plus
    # every pattern of two full 16-bit low halves around ties
    rng = np.random.default_rng(11)
    u = np.arange(0, 1 << 32, 257, dtype=np.uint64).astype(np.uint32)
    hi_words = rng.integers(0, 1 << 16, 2, dtype=np.uint64).astype(np.uint32) << 16
    u = np.concatenate([u] + [w | np.arange(1 << 16, dtype=np.uint32) for w in hi_words])
    x = u.view(np.float32)
    fin = np.isfinite(x)
    got = _bits(oracle.round_bf16(x))
    # finite inputs: the definition (a result beyond the largest BF16 is inf)
    want = _round_bf16_by_definition(x[fin])
    assert np.array_equal(got[fin], want)
    # and the library's BF16 conversion agrees on every input, NaN as NaN
    torch = pytest.importorskip("torch")
    t = torch.from_numpy(x.copy()).to(torch.bfloat16).to(torch.float32).numpy()
    nan = np.isnan(x)
    assert np.array_equal(_bits(t)[~nan], got[~nan])
    assert np.all(np.isnan(got.view(np.float32)[nan]))
