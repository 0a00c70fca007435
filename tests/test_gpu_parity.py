"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

Bars (readings of Sec. 2.1 of Burdanov, Hasler & de Wit 2023):
* nearest shifts, FP32 storage: stack values, n_cov and candidate lists are
  bit-exact with the oracle's FP32-sequential mode;
* FP16/BF16 storage: bit-exact with the FP32-sequential oracle run on the
  frames rounded to the storage type (round to nearest even), and within
  sum_i |I_i| u/2 + FP32 accumulation of the FP64 oracle on the FP32 frames;
* bilinear shifts: |S - S64| <= 1e-5 max(|S64|, sqrt(N)) per output;
* normalisation: mu, sigma within 1e-12 relative, outputs within 1 ulp.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_07293_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def ragged_field(seed=3, N=13, H=53, W=77, nv=(9, 7)):
    fr = synth.noise(N, H, W, seed=seed)
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, 3.0, N))
    f = synth.field_params(W, H, N, float(t[N // 2]), -2.1, 0.55, nv[0], -1.3, 0.45, nv[1],
                           tau=3.0)
    synth.render_movers(fr, t, f["t_ref"], [[30.0, 20.0, 1.1, -0.8, 2.5]])
    return fr, t, f


# ------------------------------------------------------------------ a1

@pytest.mark.parametrize("mode", ["nearest", "bilinear"])
def test_shift_tables_match_oracle(st, mode):
    for name, kw in [("tiny", {}), ("mid", dict(width=64, n_frames=64)),
                     ("speculoos", dict(width=64, n_frames=256))]:
        d = synth.make_field(name, **kw)
        f = d["field"]
        with st.Plan(f, mode=mode) as p:
            sx, sy, fx, fy = p.shift_tables(0, d["times"])
        osx, ofx = oracle.shift_tables(d["times"], f["t_ref"], f["vx0"], f["dvx"], f["nvx"], mode)
        osy, ofy = oracle.shift_tables(d["times"], f["t_ref"], f["vy0"], f["dvy"], f["nvy"], mode)
        assert np.array_equal(sx, osx) and np.array_equal(sy, osy), name
        if mode == "bilinear":
            assert np.array_equal(fx, ofx.astype(np.float32)), name
            assert np.array_equal(fy, ofy.astype(np.float32)), name


# ------------------------------------------------------------------ a3

def test_dump_stack_nearest_f32_bitexact(st):
    fr, t, f = ragged_field()
    ks = np.arange(f["nvx"] * f["nvy"], dtype=np.int32)
    with st.Plan(f) as p:
        S, Cv = p.dump_stack(0, dev(fr), t, ks)
    oS, oC = oracle.stack_planes(fr, t, f, ks, prec="fp32")
    assert np.array_equal(Cv.cpu().numpy(), oC)
    assert np.array_equal(S.cpu().numpy(), oS.astype(np.float32))


@pytest.mark.parametrize("name,kw", [("tiny", {}),
                                     ("mid", dict(width=192, n_frames=24, nv=33)),
                                     ("speculoos", dict(width=160, n_frames=48, nv=41))])
def test_search_nearest_f32_bitexact(st, name, kw):
    d = synth.make_field(name, **kw)
    fr = np.nan_to_num(d["frames"], nan=0.0)
    with st.Plan(d["field"]) as p:
        got = p.candidates(dev(fr), d["times"])
    ref = oracle.search(fr, d["times"], d["field"], prec="fp32")
    assert len(ref) > 0
    assert got["x"].tolist() == ref["x"].tolist()
    assert got["y"].tolist() == ref["y"].tolist()
    assert got["k"].tolist() == ref["k"].tolist()
    assert got["n_cov"].tolist() == ref["n_cov"].tolist()
    assert np.array_equal(got["stack"], ref["stack"].astype(np.float32))
    assert np.array_equal(got["snr"], ref["snr"].astype(np.float32))
    assert np.all(got["field"] == 0)


def test_search_finds_injected_movers(st):
    d = synth.make_field("tiny")
    with st.Plan(d["field"]) as p:
        got = p.candidates(dev(d["frames"]), d["times"])
    for (x0, y0, vx, vy, A) in d["truth"]:
        _, _, k = synth.velocity_index(d["field"], vx, vy)
        hit = (got["k"] == k) & (np.abs(got["x"] - x0) <= 1) & (np.abs(got["y"] - y0) <= 1)
        assert hit.any(), (x0, y0, vx, vy)


# ------------------------------------------------------------------ a7

@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_reduced_storage_bitexact_on_rounded_frames(st, storage):
    fr, t, f = ragged_field(seed=5)
    ks = np.arange(f["nvx"] * f["nvy"], dtype=np.int32)
    with st.Plan(f, storage=storage) as p:
        S, Cv = p.dump_stack(0, dev(fr), t, ks)
        got = p.candidates(dev(fr), t)
    S = S.cpu().numpy()
    rounded = fr.astype(np.float16).astype(np.float32) if storage == "f16" else \
        oracle.round_bf16(fr)
    oS, oC = oracle.stack_planes(rounded, t, f, ks, prec="fp32")
    assert np.array_equal(S, oS.astype(np.float32))
    ref = oracle.search(rounded, t, f, prec="fp32")
    assert got[["x", "y", "k"]].tolist() == ref[["x", "y", "k"]].tolist()
    # stated error against the FP64 oracle on the unrounded FP32 frames
    S64, _ = oracle.stack_planes(fr, t, f, ks, prec="fp64")
    absI, _ = oracle.stack_planes(np.abs(fr), t, f, ks, prec="fp64")
    u = 2.0 ** -11 if storage == "f16" else 2.0 ** -8   # half an ulp, relative
    N = f["n_frames"]
    bound = absI * u + N * 2.0 ** -24 * absI + 1e-30
    assert np.all(np.abs(S - S64) <= bound)


# ------------------------------------------------------------------ a4

def test_bilinear_within_tolerance_of_fp64(st):
    fr, t, f = ragged_field(seed=9)
    ks = np.arange(f["nvx"] * f["nvy"], dtype=np.int32)
    with st.Plan(f, mode="bilinear") as p:
        S, Cv = p.dump_stack(0, dev(fr), t, ks)
    oS, oC = oracle.stack_planes(fr, t, f, ks, mode="bilinear", prec="fp64")
    N = f["n_frames"]
    S = S.cpu().numpy().astype(np.float64)
    assert np.array_equal(Cv.cpu().numpy(), oC)
    assert np.all(np.abs(S - oS) <= 1e-5 * np.maximum(np.abs(oS), math.sqrt(N)))


def test_bilinear_search_candidates(st):
    d = synth.make_field("mid", width=128, n_frames=32, nv=21, n_blobs=0)
    fr, t, f = d["frames"], d["times"], d["field"]
    with st.Plan(f, mode="bilinear") as p:
        got = p.candidates(dev(fr), t)
    ref = oracle.search(fr, t, f, mode="bilinear", prec="fp64")
    # every oracle candidate clear of ties and of the threshold is found, and
    # every GPU candidate is either an oracle candidate or a near-tie
    gk = set(zip(got["x"].tolist(), got["y"].tolist(), got["k"].tolist()))
    rk = set(zip(ref["x"].tolist(), ref["y"].tolist(), ref["k"].tolist()))
    assert len(rk) > 0
    for (x, y, k) in sorted(gk ^ rk):
        # a point in one list only must be a near-tie under the stated error:
        # its S within 2e-5 max(|S|, sqrt(N)) of its threshold or of a neighbour
        nb = [(x + dx, y + dy, k) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
              if 0 <= x + dx < f["width"] and 0 <= y + dy < f["height"]]
        S64, C64 = oracle.stack_points(fr, t, f, np.array(nb, np.int32), mode="bilinear")
        c = nb.index((x, y, k))
        s = S64[c]
        tol = 2e-5 * max(abs(s), math.sqrt(f["n_frames"]))
        thr = float(np.float32(f["snr_threshold"] * math.sqrt(C64[c])))
        gaps = [abs(s - thr)] + [abs(s - S64[j]) for j in range(len(nb)) if j != c]
        assert min(gaps) <= tol, (x, y, k, s, thr)


# ------------------------------------------------------------------ a2

@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_normalize_matches_oracle(st, storage):
    d = synth.make_field("mid", width=256, n_frames=6, n_blobs=30)
    raw = d["frames"] * 3.0 + 250.0
    raw[0, 5, 7] = 1e5  # an outlier to clip
    with st.Plan(d["field"], storage=storage, normalize=True) as p:
        cube, mu, sd = p.normalize(0, dev(raw))
    omu, osd = oracle.normalize(raw)[1:]
    out, _, _ = oracle.normalize(raw)
    assert np.all(np.abs(mu - omu) <= 1e-12 * np.abs(omu))
    assert np.all(np.abs(sd - osd) <= 1e-12 * osd)
    got = cube.float().cpu().numpy()
    if storage == "f32":
        ulp = np.spacing(np.abs(out).astype(np.float32))
        assert np.all(np.abs(got - out) <= ulp)
    else:
        ref = out.astype(np.float16).astype(np.float32) if storage == "f16" else \
            oracle.round_bf16(out)
        # one FP32 ulp before rounding may move a value across a rounding boundary
        step = np.spacing(np.abs(ref).astype(np.float16 if storage == "f16" else np.float32))
        if storage == "bf16":
            step = np.abs(ref) * 2.0 ** -7 + 1e-30
        assert np.all(np.abs(got - ref) <= step)
    assert np.all(got[np.isnan(raw)] == 0.0)


def test_normalize_degenerate_frames(st):
    # a frame with no finite pixel and a constant frame have no sky scatter:
    # both normalise to zeros with the oracle's mu and sigma; the ordinary
    # frame between them is unaffected
    d = synth.make_field("tiny")
    raw = d["frames"][:3] * 2.0 + 5.0
    raw[0] = np.nan
    raw[2] = 7.25
    f = dict(d["field"], n_frames=3)
    with st.Plan(f, normalize=True) as p:
        cube, mu, sd = p.normalize(0, dev(raw))
    out, omu, osd = oracle.normalize(raw)
    got = cube.cpu().numpy()
    assert np.all(got[0] == 0.0) and np.all(got[2] == 0.0)
    assert mu[0] == omu[0] == 0.0 and sd[0] == osd[0] == 0.0
    assert mu[2] == omu[2] == 7.25 and sd[2] == osd[2] == 0.0
    assert abs(mu[1] - omu[1]) <= 1e-12 * abs(omu[1]) and abs(sd[1] - osd[1]) <= 1e-12 * osd[1]
    assert np.all(np.abs(got[1] - out[1]) <= np.spacing(np.abs(out[1]).astype(np.float32)))


def test_normalized_search_finds_movers(st):
    d = synth.make_field("mid", width=256, n_frames=32, nv=41, n_movers=6)
    raw = d["frames"] * 2.0 + 100.0
    with st.Plan(d["field"], normalize=True) as p:
        got = p.candidates(dev(raw), d["times"])
    found = 0
    for (x0, y0, vx, vy, A) in d["truth"]:
        _, _, k = synth.velocity_index(d["field"], vx, vy)
        a0, b0 = k % d["field"]["nvx"], k // d["field"]["nvx"]
        near = (np.abs(got["x"] - x0) <= 2) & (np.abs(got["y"] - y0) <= 2) & \
            (np.abs(got["k"] % d["field"]["nvx"] - a0) <= 1) & \
            (np.abs(got["k"] // d["field"]["nvx"] - b0) <= 1)
        found += bool(near.any())
    assert found >= 1


# ------------------------------------------------------------- a5/a6 rules

def test_golden_rule_fixtures_on_gpu(st):
    import json
    import os
    cases = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                        "candidate_rules.json")))["cases"]
    for case in cases:
        N, H, W = case["N"], case["H"], case["W"]
        fr = np.zeros((N, H, W), np.float32)
        for (i, x, y, v) in case["points"]:
            fr[i, y, x] = v
        vx0, dvx, nvx, vy0, dvy, nvy = case["grid"]
        f = synth.field_params(W, H, N, case["t_ref"], vx0, dvx, int(nvx), vy0, dvy, int(nvy),
                               case["tau"], case["min_coverage"])
        with st.Plan(f) as p:
            got = p.candidates(dev(fr), np.array(case["times"], np.float64))
        g = [[int(r["x"]), int(r["y"]), int(r["k"]), int(r["n_cov"]), float(r["stack"]),
              float(r["snr"])] for r in got]
        assert g == case["expected"], case["name"]


def test_overflow_reports_true_count(st):
    d = synth.make_field("tiny", tau=2.5)
    fr = dev(d["frames"])
    with st.Plan(d["field"]) as p:
        full = p.candidates(fr, d["times"])
        out, n, status = p.search(fr, d["times"], capacity=5)
        assert status == st.ST_ERR_OVERFLOW and n == len(full) and n > 5
        part = p.to_numpy(out, 5)
        assert part.tobytes() == full[:5].tobytes()
        # the plan stays usable
        again = p.candidates(fr, d["times"])
        assert again.tobytes() == full.tobytes()


def test_pending_overflow_is_an_error(st):
    d = synth.make_field("tiny", tau=0.0)
    with st.Plan(d["field"], pending_capacity=64) as p:
        with pytest.raises(st.StError) as e:
            p.search(dev(d["frames"]), d["times"], capacity=10)
        assert e.value.status == st.ST_ERR_OVERFLOW


def test_host_buffer_entry_point_matches_device(st):
    d = synth.make_field("tiny")
    with st.Plan(d["field"]) as p:
        dv = p.candidates(dev(d["frames"]), d["times"])
        hv, n = p.search_host(d["frames"], d["times"], capacity=4096)
        assert n == len(dv) and hv.tobytes() == dv.tobytes()
        assert p.last_launch_count() > 0


@pytest.mark.parametrize("W,H", [(16384, 8), (8, 16384)])
def test_search_at_the_frame_size_limits(st, W, H):
    # the largest width and height a plan accepts: coordinates near 2^14 in
    # the packed (field, k, y, x) sort key, and a grid of many tiles along
    # one axis; sources at both ends of the long axis
    N = 8
    fr = synth.noise(N, H, W, seed=40 + W % 7)
    t = np.arange(N, dtype=np.float64)
    f = synth.field_params(W, H, N, 4.0, -0.25, 0.25, 3, -0.25, 0.25, 3, tau=4.0)
    far = (W - 3, 4) if W > H else (4, H - 3)
    synth.render_movers(fr, t, 4.0, [[far[0], far[1], 0.0, 0.0, 6.0], [3.0, 3.0, 0.25, 0.0, 6.0]])
    with st.Plan(f) as p:
        got = p.candidates(dev(fr), t)
    ref = oracle.search(fr, t, f, prec="fp32")
    assert len(ref) > 0 and (ref["x"].max() >= W - 8 or ref["y"].max() >= H - 8)
    assert got[["x", "y", "k", "n_cov"]].tolist() == ref[["x", "y", "k", "n_cov"]].tolist()
    assert np.array_equal(got["stack"], ref["stack"].astype(np.float32))


def test_search_on_the_largest_grid(st):
    # nvx * nvy = 2^26, the largest grid a plan accepts (velocity indices up
    # to 2^26 - 1 in the sort key), on a small field of pure noise
    N, H, W = 8, 8, 8
    fr = synth.noise(N, H, W, seed=77)
    t = np.arange(N, dtype=np.float64)
    nv = 8192
    f = synth.field_params(W, H, N, 4.0, -0.5, 1.0 / nv, nv, -0.5, 1.0 / nv, nv, tau=4.5)
    # (every tile is an edge tile, so the kernel's pre-filter holds points to
    # the threshold at the minimum coverage: about 3400 pass it here)
    with st.Plan(f) as p:
        got = p.candidates(dev(fr), t)
    ref = oracle.search(fr, t, f, prec="fp32")
    assert len(ref) > 0 and ref["k"].max() >= 1 << 25
    assert got[["x", "y", "k", "n_cov"]].tolist() == ref[["x", "y", "k", "n_cov"]].tolist()
    assert np.array_equal(got["stack"], ref["stack"].astype(np.float32))


def test_empty_result_and_single_frame(st):
    fr = np.zeros((1, 5, 7), np.float32)
    f = synth.field_params(7, 5, 1, 0.0, -1.0, 1.0, 3, 0.0, 1.0, 1, tau=1.0)
    with st.Plan(f) as p:
        got = p.candidates(dev(fr), np.array([0.0]))
    assert len(got) == 0
