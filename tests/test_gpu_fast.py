"""GPU parity of the register-window (TMA-staged) nearest-shift stack kernel.

Same bar as the direct-gather kernel: stack values, coverage and candidate
lists bit-exact with the FP32-sequential oracle (Sec. 2.1 reading of the
search), on fields with ragged tiles (width not a multiple of 32, height not
a multiple of 16, velocity counts not multiples of 8), edge tiles, and both
signs of t - t_ref.
"""
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


VARIANTS = [0, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11]  # plan default and every FP32 register-window variant
X2_TILES = (2, 11)  # two x-velocities a thread (8 or 16 consumer warps)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def field(seed, W=96, H=45, N=19, nvx=13, nvy=11, dv=0.25, span=2.0, movers=2, ref=None):
    fr = synth.noise(N, H, W, seed=seed)
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, span, N))
    t_ref = float(t[N // 3 if ref is None else ref])
    f = synth.field_params(W, H, N, t_ref, -dv * (nvx // 2) - 0.1, dv, nvx,
                           -dv * (nvy // 2) + 0.05, dv, nvy, tau=3.5)
    mv = [[W * 0.3, H * 0.5, 1.0, -0.5, 2.5], [W * 0.7, H * 0.3, -0.75, 0.5, 3.0]][:movers]
    synth.render_movers(fr, t, f["t_ref"], mv)
    return fr, t, f


@pytest.mark.parametrize("seed,shape", [(1, dict()), (2, dict(W=128, H=64, N=40, nvx=16, nvy=16)),
                                        (3, dict(W=36, H=17, N=9, nvx=5, nvy=3)),
                                        (4, dict(W=200, H=33, N=64, nvx=24, nvy=9, dv=0.1))])
def test_fast_dump_bitexact(st, seed, shape):
    fr, t, f = field(seed, **shape)
    ks = np.arange(f["nvx"] * f["nvy"], dtype=np.int32)
    oS, oC = oracle.stack_planes(fr, t, f, ks, prec="fp32")
    for tile in VARIANTS:
        with st.Plan(f, tile=tile) as p:
            S, Cv = p.dump_stack(0, dev(fr), t, ks)
            p.candidates(dev(fr), t)
            assert p.last_stack_variant(0) == 1, "register-window kernel not used"
            if tile in X2_TILES:   # these fields' motion fits the 16-velocity boxes
                assert "_o48_" in p.stack_variant_name(0), p.stack_variant_name(0)
        assert np.array_equal(Cv.cpu().numpy(), oC), tile
        assert np.array_equal(S.cpu().numpy(), oS.astype(np.float32)), tile


def test_fast_degenerate_grids_and_frames(st):
    # one velocity at rest (the stack is the plain frame sum, Sec. 2.1's
    # zero-motion case), and a frame narrower and shorter than one tile
    N, H, W = 12, 20, 40
    fr = synth.noise(N, H, W, seed=31)
    t = np.arange(N, dtype=np.float64) * 0.3
    f0 = synth.field_params(W, H, N, float(t[5]), 0.0, 1.0, 1, 0.0, 1.0, 1, tau=2.0)
    fr2, t2, f2 = field(32, W=12, H=5, N=10, nvx=3, nvy=2)
    frame_sum = np.zeros((H, W), np.float32)
    for i in range(N):
        frame_sum = (frame_sum + fr[i]).astype(np.float32)
    for frames, times, f in ((fr, t, f0), (fr2, t2, f2)):
        ks = np.arange(f["nvx"] * f["nvy"], dtype=np.int32)
        oS, oC = oracle.stack_planes(frames, times, f, ks, prec="fp32")
        ref = oracle.search(frames, times, f, prec="fp32")
        if f is f0:
            # the single velocity at rest: the oracle's plane is the frame sum
            assert np.array_equal(oS[0].astype(np.float32), frame_sum)
        for tile in VARIANTS:
            with st.Plan(f, tile=tile) as p:
                S, Cv = p.dump_stack(0, dev(frames), times, ks)
                got = p.candidates(dev(frames), times)
                assert p.last_stack_variant(0) == 1, "register-window kernel not used"
            assert np.array_equal(Cv.cpu().numpy(), oC), tile
            assert np.array_equal(S.cpu().numpy(), oS.astype(np.float32)), tile
            if f is f0:
                assert np.array_equal(S.cpu().numpy()[0], frame_sum), tile
            assert got[["x", "y", "k", "n_cov"]].tolist() == \
                ref[["x", "y", "k", "n_cov"]].tolist(), tile


@pytest.mark.parametrize("seed,shape", [(5, dict()), (6, dict(W=256, H=80, N=48, nvx=33, nvy=17)),
                                        (7, dict(W=64, H=64, N=30, nvx=8, nvy=8, ref=-1))])
def test_fast_search_equals_generic_and_oracle(st, seed, shape):
    fr, t, f = field(seed, **shape)
    with st.Plan(f) as p:
        fast = p.candidates(dev(fr), t)
        assert p.last_stack_variant(0) == 1
    with st.Plan(f, tile=1) as p:
        gen = p.candidates(dev(fr), t)
        assert p.last_stack_variant(0) == 0
    ref = oracle.search(fr, t, f, prec="fp32")
    assert len(ref) > 0
    assert fast.tobytes() == gen.tobytes()
    assert fast[["x", "y", "k", "n_cov"]].tolist() == ref[["x", "y", "k", "n_cov"]].tolist()
    assert np.array_equal(fast["stack"], ref["stack"].astype(np.float32))


def test_fast_dense_candidates_every_row(st):
    # a low threshold puts candidates in every row and velocity slot of every
    # tile, so each output of a thread's register block is exercised
    fr, t, f = field(12, W=96, H=100, N=16, nvx=11, nvy=10)
    f = dict(f, snr_threshold=0.8)
    ref = oracle.search(fr, t, f, prec="fp32")
    assert len(ref) > 2000
    for tile in VARIANTS:
        with st.Plan(f, tile=tile) as p:
            got = p.candidates(dev(fr), t)
            assert p.last_stack_variant(0) == 1
        assert got[["x", "y", "k", "n_cov"]].tolist() == \
            ref[["x", "y", "k", "n_cov"]].tolist(), tile
        assert np.array_equal(got["stack"], ref["stack"].astype(np.float32)), tile


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_fast_reduced_storage_bitexact_on_rounded_frames(st, storage):
    fr, t, f = field(13, W=104, H=70, N=33, nvx=17, nvy=10)
    f = dict(f, snr_threshold=2.5)
    rounded = fr.astype(np.float16).astype(np.float32) if storage == "f16" else \
        oracle.round_bf16(fr)
    ks = np.arange(f["nvx"] * f["nvy"], dtype=np.int32)
    oS, oC = oracle.stack_planes(rounded, t, f, ks, prec="fp32")
    ref = oracle.search(rounded, t, f, prec="fp32")
    # 2: two x-velocities a thread; 3, 4: item loop (16 or 8 warps); 6: column pairs
    for tile in (0, 2, 3, 4, 5, 6):
        with st.Plan(f, storage=storage, tile=tile) as p:
            S, Cv = p.dump_stack(0, dev(fr), t, ks)
            got = p.candidates(dev(fr), t)
            assert p.last_stack_variant(0) == 1
            if tile == 2:
                assert "_o48_" in p.stack_variant_name(0), p.stack_variant_name(0)
        assert np.array_equal(S.cpu().numpy(), oS.astype(np.float32)), tile
        assert np.array_equal(Cv.cpu().numpy(), oC), tile
        assert got[["x", "y", "k", "n_cov"]].tolist() == \
            ref[["x", "y", "k", "n_cov"]].tolist(), tile


def test_fast_with_normalised_cube(st):
    d = synth.make_field("mid", width=192, n_frames=24, nv=33, n_movers=5)
    raw = d["frames"] * 1.5 + 40.0
    with st.Plan(d["field"], normalize=True) as p:
        fast = p.candidates(dev(raw), d["times"])
        assert p.last_stack_variant(0) == 1
    with st.Plan(d["field"], normalize=True, tile=1) as p:
        gen = p.candidates(dev(raw), d["times"])
    assert fast.tobytes() == gen.tobytes() and len(fast) > 0


def test_fast_falls_back_for_few_frames(st):
    fr, t, f = field(11, W=64, H=40, N=6, nvx=9, nvy=9)
    with st.Plan(f) as p:
        got = p.candidates(dev(fr), t)
        assert p.last_stack_variant(0) == 0
    ref = oracle.search(fr, t, f, prec="fp32")
    assert got[["x", "y", "k"]].tolist() == ref[["x", "y", "k"]].tolist()


def test_fast_falls_back_when_motion_spans_exceed_window(st):
    d = synth.make_field("tiny")   # 1 px per frame per grid step: spans too wide
    with st.Plan(d["field"]) as p:
        got = p.candidates(dev(d["frames"]), d["times"])
        assert p.last_stack_variant(0) == 0
    ref = oracle.search(d["frames"], d["times"], d["field"], prec="fp32")
    assert got[["x", "y", "k"]].tolist() == ref[["x", "y", "k"]].tolist()


def test_two_velocity_variant_at_the_edge_of_its_box(st):
    # velocity step 0.45 over |dt| up to about 2: an 8-velocity tile's column
    # offsets reach 8 (its box's limit), a 16-velocity tile's reach 16, so
    # lane 31 of some warp reads the last column of the wider box.  (With
    # FP32 storage and a uniform velocity grid a motion that fits the
    # 8-velocity box has fitted the 16-velocity one in every case tried.)
    fr, t, f = field(15, W=128, H=40, N=24, nvx=24, nvy=6, dv=0.45, span=4.0, ref=12)
    ks = np.arange(f["nvx"] * f["nvy"], dtype=np.int32)
    oS, oC = oracle.stack_planes(fr, t, f, ks, prec="fp32")
    ref = oracle.search(fr, t, f, prec="fp32")
    for tile in X2_TILES:
        with st.Plan(f, tile=tile) as p:
            S, Cv = p.dump_stack(0, dev(fr), t, ks)
            got = p.candidates(dev(fr), t)
            assert p.last_stack_variant(0) == 1, "register-window kernel not used"
            assert "_o48_" in p.stack_variant_name(0), p.stack_variant_name(0)
        assert np.array_equal(S.cpu().numpy(), oS.astype(np.float32)), tile
        assert np.array_equal(Cv.cpu().numpy(), oC), tile
        assert got[["x", "y", "k", "n_cov"]].tolist() == ref[["x", "y", "k", "n_cov"]].tolist()


def test_add_rate_probe(st):
    for var in (0, 1, 2):
        per_clk, t = st.probe_add_rate(var, 4000)
        assert 16 <= per_clk <= 1024 and t > 1.0, (var, per_clk, t)


def test_autotune_picks_a_variant_and_caches_it(st, tmp_path):
    fr, t, f = field(14, W=128, H=96, N=40, nvx=16, nvy=12)
    cache = str(tmp_path / "tune.json")
    with st.Plan(f) as p:
        ref = p.candidates(dev(fr), t)
    with st.Plan(f, tile=-1, tune_cache=cache) as p:
        got = p.candidates(dev(fr), t)
        assert p.last_stack_variant(0) == 1
    assert got.tobytes() == ref.tobytes()
    import json
    with open(cache) as fh:
        tab = json.load(fh)
    assert len(tab) == 1 and 0 <= list(tab.values())[0] < len(VARIANTS) - 1
    with st.Plan(f, tile=-1, tune_cache=cache) as p:   # served from the cache
        again = p.candidates(dev(fr), t)
    assert again.tobytes() == ref.tobytes()


def test_multi_field_plan_equals_single_field_plans(st):
    specs = [dict(seed=15, W=96, H=64, N=20, nvx=9, nvy=8),
             dict(seed=16, W=128, H=48, N=33, nvx=12, nvy=5),
             dict(seed=17, W=64, H=64, N=9, nvx=8, nvy=8)]
    fields = [field(**sp) for sp in specs]
    singles = []
    for fr, t, f in fields:
        with st.Plan(f) as p:
            singles.append(p.candidates(dev(fr), t))
    with st.Plan([f for _, _, f in fields]) as p:
        out, n, status = p.search([dev(fr) for fr, _, _ in fields], [t for _, t, _ in fields],
                                  capacity=1 << 16)
        allc = p.to_numpy(out, n)
    assert status == st.ST_OK
    for i, c in enumerate(singles):
        mine = allc[allc["field"] == i]
        assert mine[["x", "y", "k", "n_cov"]].tolist() == c[["x", "y", "k", "n_cov"]].tolist()
        assert np.array_equal(mine["stack"], c["stack"])
    assert np.all(np.diff(allc["field"]) >= 0)   # sorted by field first


@pytest.mark.parametrize("mode", ["nearest", "bilinear"])
def test_batched_fields_one_persistent_launch(st, mode):
    # uneven frame counts, sizes and grids in one plan: every field that fits
    # the register-window kernel runs in ONE persistent launch (items taken
    # longest field first); a field whose motion does not fit (wide span)
    # takes the direct-gather kernel.  Each field's candidates equal its
    # single-field plan's and, for nearest shifts, the oracle's.
    specs = [dict(seed=31, W=96, H=64, N=20, nvx=9, nvy=8),
             dict(seed=32, W=160, H=40, N=57, nvx=19, nvy=6, dv=0.12),
             dict(seed=33, W=64, H=72, N=9, nvx=8, nvy=13),
             dict(seed=34, W=128, H=33, N=41, nvx=5, nvy=17, dv=0.2, ref=-1),
             dict(seed=35, W=80, H=48, N=16, nvx=9, nvy=9, dv=2.0)]   # does not fit
    fields = [field(**sp) for sp in specs]
    singles = []
    for fr, t, f in fields:
        with st.Plan(f, mode=mode) as p:
            singles.append(p.candidates(dev(fr), t))
    with st.Plan([f for _, _, f in fields], mode=mode) as p:
        out, n, status = p.search([dev(fr) for fr, _, _ in fields], [t for _, t, _ in fields],
                                  capacity=1 << 18)
        allc = p.to_numpy(out, n)
        used = [p.last_stack_variant(i) for i in range(len(fields))]
        _, stack_launches = p.last_stack_kernel_time()
    assert status == st.ST_OK
    assert used == [1, 1, 1, 1, 0]
    assert stack_launches == 2      # one persistent launch + the direct-gather field
    for i, c in enumerate(singles):
        mine = allc[allc["field"] == i]
        assert mine.tobytes() == c.tobytes() or (
            mine[["x", "y", "k", "n_cov"]].tolist() == c[["x", "y", "k", "n_cov"]].tolist() and
            np.array_equal(mine["stack"], c["stack"])), i
        if mode == "nearest":
            fr, t, f = fields[i]
            ref = oracle.search(fr, t, f, prec="fp32")
            assert mine[["x", "y", "k", "n_cov"]].tolist() == \
                ref[["x", "y", "k", "n_cov"]].tolist(), i
    assert np.all(np.diff(allc["field"]) >= 0)
