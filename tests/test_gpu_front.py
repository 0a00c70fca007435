"""GPU parity of the pre-tracking front end (Sec. 2.1) against oracle/front.py:
median star removal, sums of every n frames and 2 x 2 binning, bit-exact
(selection and fixed-order FP32 sums), on ragged sizes, masked (NaN) samples,
odd and even frame counts, in place; plus the search it prepares: with the
stars removed the candidates are the mover's, not the stars'."""
import numpy as np
import pytest

import synth
from oracle import front

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


def cube(seed, N, H, W, nan_frac=0.02, dup=False):
    rng = np.random.default_rng(seed)
    fr = rng.normal(0.0, 1.0, (N, H, W)).astype(np.float32)
    if dup:   # many equal values: ties in the selection
        fr = np.round(fr * 2.0).astype(np.float32)
    fr[rng.random(fr.shape) < nan_frac] = np.nan
    if N > 2:
        fr[:, 0, 0] = np.nan   # a pixel masked in every frame
    return fr


@pytest.mark.parametrize("N,H,W,dup,nan_frac", [
    (1, 5, 7, False, 0.02), (2, 9, 33, False, 0.02), (7, 37, 53, False, 0.02),
    (32, 11, 13, True, 0.02), (33, 17, 19, False, 0.02), (50, 64, 96, False, 0.02),
    (64, 31, 40, True, 0.02), (257, 16, 24, False, 0.02), (768, 4, 40, False, 0.02),
    # few or no masked samples (the middle positions of the full column), and
    # many (masked samples of either parity of count, odd and even N)
    (50, 64, 96, False, 0.0), (49, 33, 40, False, 0.0), (16, 9, 40, True, 0.0),
    (64, 16, 40, False, 0.3), (63, 16, 40, True, 0.5), (3, 9, 33, False, 0.4),
    (60, 8, 64, False, 0.05)])
def test_median_subtract_bitexact(st, N, H, W, dup, nan_frac):
    fr = cube(N, N, H, W, nan_frac=nan_frac, dup=dup)
    ref, rmed = front.median_subtract(fr)
    out, med = st.median_subtract(dev(fr), with_median=True)
    torch.cuda.synchronize()
    assert np.array_equal(med.cpu().numpy(), rmed, equal_nan=True)
    assert np.array_equal(out.cpu().numpy(), ref, equal_nan=True)
    # in place
    d = dev(fr)
    st.median_subtract(d, out=d)
    assert np.array_equal(d.cpu().numpy(), ref, equal_nan=True)


def test_median_limits(st):
    with pytest.raises(st.StError):
        st.median_subtract(torch.zeros((769, 2, 4), device="cuda"))


@pytest.mark.parametrize("N,n,H,W", [(17, 5, 19, 23), (13, 13, 8, 8), (12, 1, 3, 5), (4, 7, 2, 2)])
def test_sum_frames_bitexact(st, N, n, H, W):
    fr = cube(100 + N, N, H, W)
    t = np.cumsum(np.random.default_rng(N).uniform(0.5, 1.5, N))
    ref, rt = front.sum_frames(fr, t, n)
    out, tout = st.sum_frames(dev(fr), t, n)
    torch.cuda.synchronize()
    assert out.shape[0] == ref.shape[0] == N // n
    assert np.array_equal(out.cpu().numpy(), ref, equal_nan=True)
    assert np.array_equal(tout, rt)


@pytest.mark.parametrize("N,H,W", [(3, 7, 9), (2, 64, 128), (1, 1, 5), (5, 33, 2)])
def test_bin2x2_bitexact(st, N, H, W):
    fr = cube(200 + H, N, H, W, nan_frac=0.0)
    ref = front.bin2x2(fr)
    out = st.bin2x2(dev(fr))
    torch.cuda.synchronize()
    assert tuple(out.shape) == ref.shape
    assert np.array_equal(out.cpu().numpy(), ref, equal_nan=True)


def test_star_removal_then_search_finds_the_mover(st):
    # a field of bright static stars over noise plus one mover: searched
    # as is, the stars dominate the candidates; after the median removal the
    # mover is the brightest detection at its own velocity
    d = synth.make_field("mid", width=192, n_frames=32, nv=21, n_movers=0, n_blobs=0, tau=6.0)
    f, t, fr = d["field"], d["times"], d["frames"].copy()
    m = [96.3, 80.2, 2.0, -1.5, 3.0]            # x0, y0 at t_ref, vx, vy (px/h), amplitude
    synth.render_movers(fr, t, f["t_ref"], [m])
    rng = np.random.default_rng(3)
    yy, xx = np.mgrid[0:192, 0:192]
    for _ in range(30):
        x0, y0, a = rng.uniform(10, 182), rng.uniform(10, 182), rng.uniform(20, 200)
        fr += (a * np.exp(-((xx - x0) ** 2 + (yy - y0) ** 2) / 4.0)).astype(np.float32)[None]
    a_t, b_t, k_t = synth.velocity_index(f, m[2], m[3])
    with st.Plan(f, normalize=False) as p:
        raw = p.candidates(dev(fr), t)
    clean = st.median_subtract(dev(fr))
    with st.Plan(f, normalize=False) as p:
        got = p.candidates(clean, t)
    assert len(raw) > 5 * max(len(got), 1)      # stars swamp the raw search
    best = got[np.argmax(got["snr"])]
    assert abs(best["x"] - m[0]) <= 2 and abs(best["y"] - m[1]) <= 2
    assert abs(int(best["k"]) % f["nvx"] - a_t) <= 1 and abs(int(best["k"]) // f["nvx"] - b_t) <= 1
