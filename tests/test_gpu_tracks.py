"""GPU parity of the linking of detections into tracks (oracle/tracks.py):
the components, representatives and sizes of st_link_tracks equal the
oracle's on real search outputs (several fields, dense detections), speed
and position angle within FP32 rounding of the oracle's FP64 values; an
injected mover becomes one track at its own velocity."""
import math

import numpy as np
import pytest

import synth
from oracle import tracks as otracks

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_07293_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


def grids(fields):
    return [(f["vx0"], f["dvx"], f["nvx"], f["vy0"], f["dvy"], f["nvy"]) for f in fields]


def compare(got, ref):
    assert len(got) == len(ref)
    for g, r in zip(got, ref):
        for key in ("x", "y", "k", "field", "n_cov", "members"):
            assert int(g[key]) == r[key], (key, g, r)
        assert g["snr"] == np.float32(r["snr"]) and g["stack"] == np.float32(r["stack"])
        for key in ("vx", "vy", "speed"):
            assert abs(float(g[key]) - r[key]) <= 1e-6 * max(1.0, abs(r[key]))
        dpa = abs(float(g["pa"]) - r["pa"])
        assert min(dpa, 360.0 - dpa) <= 1e-4


@pytest.mark.parametrize("r_xy,r_v", [(2, 1), (1, 0), (3, 2)])
def test_tracks_equal_oracle(st, r_xy, r_v):
    ds = [synth.make_field("mid", seed=500 + j, width=160 + 32 * j, n_frames=20 + 4 * j,
                           nv=13 + 2 * j, n_movers=4, n_blobs=0, tau=3.0) for j in range(3)]
    fields = [d["field"] for d in ds]
    with st.Plan(fields) as p:
        out, n, s = p.search([torch.from_numpy(d["frames"]).cuda() for d in ds],
                             [d["times"] for d in ds], capacity=1 << 18)
        assert s == st.ST_OK and n > 1000
        cand = p.to_numpy(out, n)
        got = p.link_tracks(out[:n], n, r_xy=r_xy, r_v=r_v)
    ref = otracks.link_tracks(cand, grids(fields), r_xy=r_xy, r_v=r_v)
    compare(got, ref)
    assert sum(int(t["members"]) for t in got) == n


def test_mover_is_one_track(st):
    d = synth.make_field("mid", seed=77, width=192, n_frames=40, nv=21, n_movers=0, n_blobs=0,
                         tau=6.0)
    f, t, fr = d["field"], d["times"], d["frames"].copy()
    m = [90.4, 101.7, -2.5, 1.0, 3.0]
    synth.render_movers(fr, t, f["t_ref"], [m])
    with st.Plan(f) as p:
        out, n, _ = p.search(torch.from_numpy(fr).cuda(), t, capacity=1 << 16)
        trk = p.link_tracks(out[:n], n)
    best = trk[np.argmax(trk["snr"])]
    assert abs(best["x"] - m[0]) <= 2 and abs(best["y"] - m[1]) <= 2
    assert abs(best["vx"] - m[2]) <= f["dvx"] and abs(best["vy"] - m[3]) <= f["dvy"]
    assert best["members"] > 1
    assert abs(best["speed"] - math.hypot(best["vx"], best["vy"])) < 1e-5
