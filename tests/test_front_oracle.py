"""Pins of the front-end oracle (oracle/front.py): closed forms for the median
combination (distinct-value permutations, NaN-masked pixels, a stationary
source under a moving one), the sums of every n frames, 2 x 2 binning of a
ramp, and the group rule (Sec. 2.1)."""
import numpy as np

from oracle import front


def test_median_of_permutations_odd_even_and_masked():
    rng = np.random.default_rng(0)
    for M in (7, 8, 31, 50):
        H, W = 3, 5
        fr = np.stack([rng.permutation(np.arange(1, M + 1)) for _ in range(H * W)], axis=1)
        fr = fr.reshape(M, H, W).astype(np.float32)
        _, med = front.median_subtract(fr)
        expect = (M + 1) / 2.0                      # odd: middle; even: mean of two middles
        assert np.all(med == np.float32(expect))
    # masked samples are excluded: values 1..9 with three of them NaN
    v = np.arange(1, 10, dtype=np.float32)
    v[[0, 4, 8]] = np.nan                           # remaining 2,3,4,6,7,8 -> (4+6)/2
    out, med = front.median_subtract(v.reshape(9, 1, 1))
    assert med[0, 0] == np.float32(5.0)
    assert np.isnan(out[0, 0, 0]) and out[1, 0, 0] == np.float32(-3.0)
    # a pixel masked in every frame stays masked
    _, med = front.median_subtract(np.full((4, 1, 2), np.nan, np.float32))
    assert np.all(np.isnan(med))


def test_median_removes_a_stationary_source_under_a_mover():
    # star pattern S plus a mover that visits each pixel in fewer than half
    # of the frames: the median is S exactly, the residual the mover alone
    N, H, W = 11, 16, 20
    yy, xx = np.mgrid[0:H, 0:W]
    # integer-valued so that (S + m) - S is exact in FP32
    S = np.round(100.0 * np.exp(-((xx - 9) ** 2 + (yy - 7) ** 2) / 4.0) + 3.0).astype(np.float32)
    fr = np.repeat(S[None], N, axis=0).copy()
    mover = np.zeros_like(fr)
    for i in range(N):
        mover[i, 2 + i % 12, i] = 50.0 + i         # one pixel per frame, never revisited
    out, med = front.median_subtract(fr + mover)
    assert np.array_equal(med, S)
    assert np.array_equal(out, ((fr + mover) - S[None]).astype(np.float32))
    assert np.array_equal(out, mover)


def test_sum_frames_closed_forms():
    N, H, W = 17, 2, 3
    fr = np.stack([np.full((H, W), i, np.float32) for i in range(N)])
    t = np.arange(N, dtype=np.float64) * 0.5
    out, tout = front.sum_frames(fr, t, 5)
    assert out.shape == (3, H, W)                   # 17 = 3 x 5 + 2 dropped
    for m in range(3):
        assert np.all(out[m] == np.float32(sum(range(5 * m, 5 * m + 5))))
        assert tout[m] == np.mean(t[5 * m:5 * m + 5])
    c = np.full((6, 2, 2), 0.25, np.float32)
    out, _ = front.sum_frames(c, np.arange(6.0), 3)
    assert np.all(out == np.float32(0.75))
    nanfr = np.zeros((4, 1, 1), np.float32)
    nanfr[1] = np.nan
    out, _ = front.sum_frames(nanfr, np.arange(4.0), 2)
    assert np.isnan(out[0, 0, 0]) and out[1, 0, 0] == 0.0


def test_bin2x2_ramp_closed_form_and_odd_edges():
    N, H, W = 2, 7, 9
    a, b, c = 0.5, -2.0, 3.0
    yy, xx = np.mgrid[0:H, 0:W]
    fr = np.repeat((a * xx + b * yy + c).astype(np.float32)[None], N, axis=0)
    out = front.bin2x2(fr)
    assert out.shape == (N, 3, 4)
    Y, X = np.mgrid[0:3, 0:4]
    expect = a * (2 * (2 * X) + 2 * (2 * X + 1)) + b * (2 * (2 * Y) + 2 * (2 * Y + 1)) + 4 * c
    assert np.array_equal(out[0], expect.astype(np.float32))
    assert np.array_equal(out[1], expect.astype(np.float32))


def test_group_rule_and_ranges():
    # 2048 px field, fastest speed 100 px/h, 50 s cadence: the group may last
    # 2048 / (0.7 * 100) = 29.26 h -> 2106 frames; at 1000 px/h -> 210 frames
    assert front.group_size(2048, 100.0, 50.0 / 3600.0) == 2106
    assert front.group_size(2048, 1000.0, 50.0 / 3600.0) == 210
    assert front.group_ranges(10, 20, 2) == [(0, 10)]
    assert front.group_ranges(100, 50, 5) == [(0, 50), (45, 95), (50, 100)]
    r = front.group_ranges(256, 50, 5)
    assert r[0] == (0, 50) and r[-1] == (206, 256)
    assert all(e - s == 50 for s, e in r)
    assert all(r[k + 1][0] <= r[k][1] - 5 for k in range(len(r) - 1))   # overlaps >= 5
