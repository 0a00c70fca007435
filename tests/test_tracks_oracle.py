"""Pins of the track-linking oracle (oracle/tracks.py): hand-built detection
sets with known components (separation, transitive chains, field and
velocity boundaries, S/N ties) and closed-form speed / position angle."""
import math

import numpy as np

from oracle import tracks

DT = np.dtype([("x", np.int32), ("y", np.int32), ("k", np.int32), ("field", np.int32),
               ("stack", np.float32), ("snr", np.float32), ("n_cov", np.int32)])
GRID = (-2.0, 1.0, 5, -2.0, 1.0, 5)   # a, b in 0..4 -> v in -2..2


def det(rows):
    a = np.array([tuple(r) for r in rows], dtype=DT)
    key = (a["field"].astype(np.int64) << 56) | (a["k"].astype(np.int64) << 30) | \
          (a["y"].astype(np.int64) << 15) | a["x"].astype(np.int64)
    return a[np.argsort(key, kind="stable")]


def k_of(a, b):
    return b * 5 + a


def test_components_transitivity_and_boundaries():
    rows = [
        # track 1: a chain x = 10, 12, 14 at one velocity (10 and 14 are 4 px apart)
        (10, 20, k_of(2, 2), 0, 9.0, 5.0, 10), (12, 20, k_of(2, 2), 0, 10.0, 6.0, 10),
        (14, 20, k_of(2, 2), 0, 8.0, 5.5, 10),
        # joined to it through a diagonal velocity neighbour (da = db = 1)
        (15, 21, k_of(3, 3), 0, 11.0, 7.0, 10),
        # two velocity steps away: not linked (r_v = 1)
        (12, 20, k_of(4, 2), 0, 20.0, 9.0, 10),
        # three pixels away in y: not linked (r_xy = 2)
        (12, 23, k_of(2, 2), 0, 7.0, 4.0, 10),
        # another field at the same place: never linked
        (12, 20, k_of(2, 2), 1, 12.0, 6.5, 10),
    ]
    c = det(rows)
    t = tracks.link_tracks(c, [GRID, GRID])
    sizes = sorted(tr["members"] for tr in t)
    assert sizes == [1, 1, 1, 4]
    big = [tr for tr in t if tr["members"] == 4][0]
    assert (big["x"], big["y"], big["snr"]) == (15, 21, 7.0)   # highest S/N member
    # tracks follow their first detection in (field, k, y, x) order: the chain
    # (first member at k = 12, y = 20) precedes the lone detections at
    # (k = 12, y = 23) and (k = 14, y = 20), then field 1
    assert [(tr["field"], tr["members"]) for tr in t] == [(0, 4), (0, 1), (0, 1), (1, 1)]
    assert [(tr["k"], tr["y"]) for tr in t[1:3]] == [(k_of(2, 2), 23), (k_of(4, 2), 20)]


def test_snr_tie_takes_the_first_detection():
    c = det([(5, 5, k_of(1, 1), 0, 3.0, 5.0, 4), (6, 5, k_of(1, 1), 0, 3.0, 5.0, 4)])
    t = tracks.link_tracks(c, [GRID])
    assert len(t) == 1 and t[0]["members"] == 2 and t[0]["x"] == 5


def test_speed_and_position_angle():
    cases = [((2, 1), 0.0), ((1, 2), 90.0), ((2, 3), 180.0), ((3, 2), 270.0), ((1, 1), 45.0)]
    for (a, b), pa in cases:
        c = det([(30, 30, k_of(a, b), 0, 1.0, 6.0, 3)])
        tr = tracks.link_tracks(c, [GRID])[0]
        vx, vy = -2.0 + a, -2.0 + b
        assert (tr["vx"], tr["vy"]) == (vx, vy)
        assert tr["speed"] == math.hypot(vx, vy)
        assert abs(tr["pa"] - pa) < 1e-12
