"""GPU parity of the register-window kernel with bilinear sampling (row a4).

The register-window kernel forms each bilinear sample in factored form (the
warp's horizontal interpolation shared by its 4 y-velocities, then two fused
multiply-adds), the direct-gather kernel as four weighted taps; both are held
to the stated bar against the FP64 oracle, |S - S64| <= 1e-5 max(|S64|,
sqrt(N)), with exact coverage.  Candidate lists must equal the direct-gather
kernel's exactly: the local-maximum resolver re-forms every reported value
with one arithmetic, and the register-window pre-filter keeps a margin.
Fields have ragged tiles, edge tiles, both signs of t - t_ref and fractional
shifts; integer shifts reduce bilinear to nearest bit for bit (Sec. 2.1
reading).
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


TILES = [0, 2, 3, 4]   # plan default and the bilinear register-window variants


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def field(seed, W=96, H=45, N=19, nvx=13, nvy=11, dv=0.2, span=2.0, ref=None, tau=3.5):
    fr = synth.noise(N, H, W, seed=seed)
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, span, N))
    t_ref = float(t[N // 3 if ref is None else ref])
    f = synth.field_params(W, H, N, t_ref, -dv * (nvx // 2) - 0.13, dv, nvx,
                           -dv * (nvy // 2) + 0.07, dv, nvy, tau=tau)
    synth.render_movers(fr, t, f["t_ref"], [[W * 0.3, H * 0.5, 0.9, -0.45, 2.5],
                                            [W * 0.7, H * 0.3, -0.7, 0.55, 3.0]])
    return fr, t, f


SHAPES = [(21, dict()), (22, dict(W=128, H=64, N=40, nvx=16, nvy=16)),
          (23, dict(W=36, H=17, N=9, nvx=5, nvy=3)),
          (24, dict(W=200, H=33, N=64, nvx=24, nvy=9, dv=0.1, ref=-1))]


@pytest.mark.parametrize("seed,shape", SHAPES)
def test_bilinear_fast_dump_equals_generic_and_fp64(st, seed, shape):
    fr, t, f = field(seed, **shape)
    ks = np.arange(f["nvx"] * f["nvy"], dtype=np.int32)
    with st.Plan(f, mode="bilinear", tile=1) as p:
        gS, gC = p.dump_stack(0, dev(fr), t, ks)
    gS, gC = gS.cpu().numpy(), gC.cpu().numpy()
    oS, oC = oracle.stack_planes(fr, t, f, ks, mode="bilinear", prec="fp64")
    N = f["n_frames"]
    assert np.array_equal(gC, oC)
    assert np.all(np.abs(gS - oS) <= 1e-5 * np.maximum(np.abs(oS), math.sqrt(N)))
    for tile in TILES:
        with st.Plan(f, mode="bilinear", tile=tile) as p:
            S, Cv = p.dump_stack(0, dev(fr), t, ks)
            p.candidates(dev(fr), t)
            assert p.last_stack_variant(0) == 1, "register-window kernel not used"
        S = S.cpu().numpy().astype(np.float64)
        assert np.array_equal(Cv.cpu().numpy(), oC), tile
        assert np.all(np.abs(S - oS) <= 1e-5 * np.maximum(np.abs(oS), math.sqrt(N))), tile


@pytest.mark.parametrize("seed,shape,tau", [(25, dict(), 3.5),
                                            (26, dict(W=256, H=80, N=48, nvx=33, nvy=17), 3.5),
                                            (27, dict(W=96, H=100, N=16, nvx=11, nvy=10), 0.8)])
def test_bilinear_fast_search_equals_generic(st, seed, shape, tau):
    # tau = 0.8 puts candidates in every row and velocity slot of every tile
    fr, t, f = field(seed, tau=tau, **shape)
    with st.Plan(f, mode="bilinear", tile=1) as p:
        gen = p.candidates(dev(fr), t)
        assert p.last_stack_variant(0) == 0
    assert len(gen) > (2000 if tau < 1 else 0)
    for tile in TILES:
        with st.Plan(f, mode="bilinear", tile=tile) as p:
            fast = p.candidates(dev(fr), t)
            assert p.last_stack_variant(0) == 1
        assert fast.tobytes() == gen.tobytes(), tile


def test_bilinear_fast_candidates_against_fp64_oracle(st):
    # every list difference with the FP64 oracle is a near-tie under the bar
    fr, t, f = field(28, W=160, H=72, N=24, nvx=17, nvy=13)
    with st.Plan(f, mode="bilinear") as p:
        got = p.candidates(dev(fr), t)
        assert p.last_stack_variant(0) == 1
    ref = oracle.search(fr, t, f, mode="bilinear", prec="fp64")
    assert len(ref) > 0
    gk = set(zip(got["x"].tolist(), got["y"].tolist(), got["k"].tolist()))
    rk = set(zip(ref["x"].tolist(), ref["y"].tolist(), ref["k"].tolist()))
    for (x, y, k) in sorted(gk ^ rk):
        nb = [(x + dx, y + dy, k) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
              if 0 <= x + dx < f["width"] and 0 <= y + dy < f["height"]]
        S64, C64 = oracle.stack_points(fr, t, f, np.array(nb, np.int32), mode="bilinear")
        c = nb.index((x, y, k))
        tol = 2e-5 * max(abs(S64[c]), math.sqrt(f["n_frames"]))
        thr = float(np.float32(f["snr_threshold"] * math.sqrt(C64[c])))
        gaps = [abs(S64[c] - thr)] + [abs(S64[c] - S64[j]) for j in range(len(nb)) if j != c]
        assert min(gaps) <= tol, (x, y, k)


def test_bilinear_fast_integer_shifts_equal_nearest(st):
    # integer times and integer velocities: every fraction is 0, so the
    # bilinear stack is the nearest stack (the special case of Sec. 2.1's
    # sub-pixel motion that reduces to whole-pixel shifts) — including the
    # coverage of samples on the last row and column
    # (dt in {-1, 0, 1} keeps the motion spans within the register window)
    N, H, W = 12, 40, 72
    fr = synth.noise(N, H, W, seed=29)
    t = np.tile([0.0, 1.0, 2.0], N // 3)
    f = synth.field_params(W, H, N, 1.0, -2.0, 1.0, 5, -3.0, 1.0, 7, tau=3.0)
    ks = np.arange(5 * 7, dtype=np.int32)
    with st.Plan(f, mode="bilinear") as p:
        bS, bC = p.dump_stack(0, dev(fr), t, ks)
        bl = p.candidates(dev(fr), t)
        assert p.last_stack_variant(0) == 1
    with st.Plan(f) as p:
        nS, nC = p.dump_stack(0, dev(fr), t, ks)
        ne = p.candidates(dev(fr), t)
    assert np.array_equal(bC.cpu().numpy(), nC.cpu().numpy())
    # fx = fy = 0: h = I exactly and fma(1, h, acc) then fma(0, ., acc) == acc + I
    assert np.array_equal(bS.cpu().numpy(), nS.cpu().numpy())
    assert bl.tobytes() == ne.tobytes()


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_bilinear_fast_reduced_storage(st, storage):
    fr, t, f = field(30, W=104, H=70, N=33, nvx=17, nvy=10, tau=2.5)
    ks = np.arange(f["nvx"] * f["nvy"], dtype=np.int32)
    with st.Plan(f, mode="bilinear", storage=storage, tile=1) as p:
        gS, gC = p.dump_stack(0, dev(fr), t, ks)
        gen = p.candidates(dev(fr), t)
    with st.Plan(f, mode="bilinear", storage=storage) as p:
        S, Cv = p.dump_stack(0, dev(fr), t, ks)
        got = p.candidates(dev(fr), t)
        assert p.last_stack_variant(0) == 1
    assert np.array_equal(Cv.cpu().numpy(), gC.cpu().numpy())
    assert got.tobytes() == gen.tobytes()
    # against FP64 on the rounded frames: FP32 accumulation error only
    rounded = fr.astype(np.float16).astype(np.float32) if storage == "f16" else \
        oracle.round_bf16(fr)
    oS, _ = oracle.stack_planes(rounded, t, f, ks, mode="bilinear", prec="fp64")
    N = f["n_frames"]
    assert np.all(np.abs(S.cpu().numpy() - oS) <= 1e-5 * np.maximum(np.abs(oS), math.sqrt(N)))
