"""Oracle of the pre-tracking front end (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module.  Plain numpy restatements, in the order the
paper gives the steps (Burdanov, Hasler & de Wit 2023, Sec. 2.1):

* median combination per group of frames, subtracted from every frame of the
  group to remove the high-S/N stationary sources (stars);
* summing of every n consecutive frames (slow movers, archival data);
* 2 x 2 spatial binning (fast movers);
* slightly overlapping groups of frames (fast movers).

Readings where the paper is silent: the median is taken over the finite
values of a pixel (NaN marks a masked pixel); an even count takes the mean
of the two middle values, formed in FP32 as (a + b) * 0.5; a pixel with no
finite value stays NaN.  Sums run in frame order with one FP32 accumulator
(NaN propagates); a trailing group shorter than n is dropped, so every
summed frame has the same exposure, and its time stamp is the FP64 mean of
the group's stamps.  Binning sums the 2 x 2 block in the fixed order
((p00 + p01) + p10) + p11 (flux kept), dropping an odd last row / column.
"""
import numpy as np


def median_subtract(frames):
    """I_i - median_j I_j per pixel (FP32), median over finite values."""
    fr = np.ascontiguousarray(frames, dtype=np.float32)
    N = fr.shape[0]
    flat = fr.reshape(N, -1)
    med = np.full(flat.shape[1], np.nan, np.float32)
    for p in range(flat.shape[1]):
        v = flat[:, p]
        v = np.sort(v[np.isfinite(v)])           # ascending, exact FP32 values
        n = len(v)
        if n == 0:
            continue
        if n % 2 == 1:
            med[p] = v[n // 2]
        else:
            med[p] = (np.float32(v[n // 2 - 1]) + np.float32(v[n // 2])) * np.float32(0.5)
    return (flat - med[None, :]).reshape(fr.shape).astype(np.float32), med.reshape(fr.shape[1:])


def sum_frames(frames, times, n):
    """Sums of every n consecutive frames (FP32, frame order) and the mean
    time stamp of each group (FP64); a trailing partial group is dropped."""
    fr = np.ascontiguousarray(frames, dtype=np.float32)
    t = np.asarray(times, dtype=np.float64)
    M = fr.shape[0] // n
    out = np.zeros((M,) + fr.shape[1:], np.float32)
    tout = np.zeros(M, np.float64)
    for m in range(M):
        acc = np.zeros(fr.shape[1:], np.float32)
        ts = 0.0
        for i in range(m * n, m * n + n):
            acc = (acc + fr[i]).astype(np.float32)
            ts += t[i]
        out[m] = acc
        tout[m] = ts / n
    return out, tout


def bin2x2(frames):
    """((p00 + p01) + p10) + p11 over 2 x 2 blocks (FP32)."""
    fr = np.ascontiguousarray(frames, dtype=np.float32)
    N, H, W = fr.shape
    h, w = H // 2, W // 2
    f = fr[:, :2 * h, :2 * w]
    p00, p01 = f[:, 0::2, 0::2], f[:, 0::2, 1::2]
    p10, p11 = f[:, 1::2, 0::2], f[:, 1::2, 1::2]
    return (((p00 + p01).astype(np.float32) + p10).astype(np.float32) + p11).astype(np.float32)


def group_size(field_px, v_max, cadence, presence=0.7):
    """Frames per group so that an object at the fastest searched speed v_max
    (px per time unit), crossing field_px pixels, is present in the group for
    `presence` of its duration: the group spans at most
    field_px / (presence * v_max), i.e. that many time units over the cadence."""
    return max(1, int(np.floor(field_px / (presence * v_max * cadence))))


def group_ranges(n_frames, size, overlap):
    """[start, end) frame ranges of groups of `size` frames, consecutive
    groups sharing `overlap` frames; the last group ends at the last frame
    (it may start earlier to keep its full size)."""
    if n_frames <= size:
        return [(0, n_frames)]
    step = size - overlap
    out = []
    s = 0
    while True:
        if s + size >= n_frames:
            out.append((max(0, n_frames - size), n_frames))
            break
        out.append((s, s + size))
        s += step
    return out
