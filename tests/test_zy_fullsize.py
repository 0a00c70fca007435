"""Parity at the headline size: one 2048^2 field of 256 frames (50 s cadence,
cosmic rays, 100 movers) and the 801 x 801 velocity grid (+-100 px/h, step
0.25 px/h), searched with the options the benchmark times: FP32 storage,
nearest shifts, the autotuned register-window variant in one persistent
launch.

The oracle cannot search all 641 601 velocity planes inside a test, so it
checks what it can compute at this size, against the bars of the small-size
parity tests (readings of Sec. 2.1 of Burdanov, Hasler & de Wit 2023):

* whole planes: the GPU's candidates in runs of four consecutive velocity
  planes (through three injected movers, the grid's first and last planes,
  where coverage is partial over much of the field, and two random runs)
  equal the oracle's list for those planes bit for bit;
* sampled candidates: 2000 reported candidates re-evaluated point by point
  by the oracle's rule (``oracle.candidates_at``): each is a candidate, with
  the same stack, coverage and S/N bit for bit;
* mover windows: around every injected mover (+-2 px, +-1 grid step in each
  velocity axis) the GPU's candidates equal the oracle's, point by point;
* the same checks with FP16 frame storage, against the oracle on the frames
  rounded to FP16;
* front end (the benchmark's configuration: median removal over groups of
  50 frames overlapping by 5, sums of every 13 frames, 2 x 2 binning): sums
  and binning compared whole, medians on 20000 sampled pixels of every
  group, bit for bit;
* refinement: 4096 candidates on the 2048^2 x 300-frame field, 128 of them
  against the FP64 oracle (J, S/N, adjoint) with the small-size bars plus
  the derived effect of the FP32 shift at shifts of up to 208 px;
* the 1024^2 x 64-frame field with its 161^2 grid, nearest (as above, for
  FP32 storage and for FP16 / BF16 storage against the oracle on the frames
  rounded to the storage type) and
  bilinear (values within 1e-5 max(|S64|, sqrt N) of the FP64 oracle, list
  differences only at near-ties);
* the multi-night workload at its full size, bit for bit;
* four fields of the 24-field batch at their full sizes in one plan (FP16
  storage, CUDA graph, one persistent launch), each against the oracle on
  its frames rounded to FP16, bit for bit;
* normalisation of the raw cube: sigma within 1e-12 relative, mu within
  1e-12 sigma (the noise frames have no sky level, so mu is near zero), and
  every output within 1 ulp of the oracle's or 1e-12 in sigma units (an
  output where the raw value and mu nearly cancel is set by the last bits
  of the FP64 mean).

The oracle normalises the raw frames (with the cosmic-ray clip at 10 sigma)
and the GPU search runs on that cube, so both sides stack the same input.
The file is named to be collected last: it takes a few minutes.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

CR_CLIP = 10.0
RUN = 4          # planes per run
N_POINTS = 2000  # sampled candidates


@pytest.fixture(scope="module")
def st():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_07293_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


@pytest.fixture(scope="module")
def field():
    d = synth.make_field("speculoos")
    cube, mu, sd = oracle.normalize(d["frames"], cr_clip=CR_CLIP)
    return d, cube, mu, sd


@pytest.fixture(scope="module")
def found(st, field):
    d, cube, _, _ = field
    frames = torch.from_numpy(cube).cuda()
    with st.Plan(d["field"], storage="f32", mode="nearest", tile=-1,
                 pending_capacity=1 << 24) as p:
        got = p.candidates(frames, d["times"], capacity=1 << 22)
        used = p.last_stack_variant(0)
    del frames
    torch.cuda.empty_cache()
    return got, used


def _key(x, y, k):
    return (np.asarray(k, np.int64) << 30) | (np.asarray(y, np.int64) << 15) | \
        np.asarray(x, np.int64)


def plane_runs(d, seed=11):
    """Starts of the runs of RUN consecutive velocity planes checked whole."""
    f = d["field"]
    nk = f["nvx"] * f["nvy"]
    starts = [0, nk - RUN]
    for m in d["truth"][:3]:
        _, _, k = synth.velocity_index(f, m[2], m[3])
        starts.append(int(min(max(k - 1, 0), nk - RUN)))
    rng = np.random.default_rng(seed)
    starts += [int(s) for s in rng.integers(0, nk - RUN, size=2)]
    return sorted(set(starts))


def check_planes(got, cube, d, starts):
    """The GPU's candidates in each run of planes equal the oracle's."""
    total = 0
    for k0 in starts:
        ref = oracle.search(cube, d["times"], d["field"], prec="fp32", k_begin=k0,
                            k_end=k0 + RUN)
        sel = got[(got["k"] >= k0) & (got["k"] < k0 + RUN)]
        assert len(sel) == len(ref), (k0, len(sel), len(ref))
        for key in ("x", "y", "k", "n_cov"):
            assert np.array_equal(sel[key], ref[key]), (k0, key)
        assert np.array_equal(sel["stack"], ref["stack"].astype(np.float32)), k0
        assert np.array_equal(sel["snr"], ref["snr"].astype(np.float32)), k0
        total += len(ref)
    return total


def check_points(got, cube, d, n_points=N_POINTS, seed=5):
    """Sampled candidates re-evaluated point by point by the oracle's rule."""
    rng = np.random.default_rng(seed)
    c = got[np.sort(rng.choice(len(got), min(n_points, len(got)), replace=False))]
    xyk = np.stack([c["x"], c["y"], c["k"]], axis=1)
    ok, S, Cv, snr = oracle.candidates_at(cube, d["times"], d["field"], xyk, prec="fp32")
    assert np.all(ok)
    assert np.array_equal(c["stack"], S.astype(np.float32))
    assert np.array_equal(c["n_cov"], Cv)
    assert np.array_equal(c["snr"], snr.astype(np.float32))
    return len(c)


def window_points(d, r_xy=2, r_v=1):
    """Every (x, y, k) within r_xy px of an injected mover's position at t_ref
    and r_v grid steps of its velocity, in (k, y, x) order, and the number of
    movers with a window."""
    f = d["field"]
    W, H, nvx, nvy = f["width"], f["height"], f["nvx"], f["nvy"]
    pts = set()
    for m in d["truth"]:
        a, b, _ = synth.velocity_index(f, m[2], m[3])
        x0, y0 = int(round(m[0])), int(round(m[1]))
        for bb in range(max(b - r_v, 0), min(b + r_v, nvy - 1) + 1):
            for aa in range(max(a - r_v, 0), min(a + r_v, nvx - 1) + 1):
                for y in range(max(y0 - r_xy, 0), min(y0 + r_xy, H - 1) + 1):
                    for x in range(max(x0 - r_xy, 0), min(x0 + r_xy, W - 1) + 1):
                        pts.add((x, y, bb * nvx + aa))
    return np.array(sorted(pts, key=lambda p: (p[2], p[1], p[0])), np.int64).reshape(-1, 3)


def check_windows(got, cube, d, pts):
    """The GPU's candidates among pts equal the oracle's, point by point;
    returns how many there are."""
    ok, S, Cv, snr = oracle.candidates_at(cube, d["times"], d["field"], pts, prec="fp32")
    want = pts[ok]
    sel = got[np.isin(_key(got["x"], got["y"], got["k"]), _key(pts[:, 0], pts[:, 1], pts[:, 2]))]
    assert np.array_equal(_key(sel["x"], sel["y"], sel["k"]),
                          _key(want[:, 0], want[:, 1], want[:, 2]))
    assert np.array_equal(sel["stack"], S[ok].astype(np.float32))
    assert np.array_equal(sel["n_cov"], Cv[ok])
    assert np.array_equal(sel["snr"], snr[ok].astype(np.float32))
    return len(want)


def test_fullsize_search_planes_and_sampled_candidates(st, field, found):
    d, cube, _, _ = field
    got, used = found
    assert used == 1, "the headline field must run on the register-window kernel"
    assert len(got) > 0 and np.all(got["field"] == 0)
    assert np.all(np.diff(_key(got["x"], got["y"], got["k"])) > 0), \
        "candidates sorted by (k, y, x), without duplicates"
    assert check_planes(got, cube, d, plane_runs(d)) > 0
    assert check_points(got, cube, d) == min(N_POINTS, len(got))


def test_fullsize_fp16_storage(st, field):
    # the headline search with FP16 frame storage (the plan rounds the cube
    # to FP16, the sums stay FP32 in frame order): bit for bit with the
    # oracle on the frames rounded to FP16, on plane runs, sampled candidates
    # and mover windows
    d, cube, _, _ = field
    frames = torch.from_numpy(cube).cuda()
    with st.Plan(d["field"], storage="f16", mode="nearest", tile=-1,
                 pending_capacity=1 << 24) as p:
        got = p.candidates(frames, d["times"], capacity=1 << 22)
        assert p.last_stack_variant(0) == 1
    del frames
    torch.cuda.empty_cache()
    r16 = cube.astype(np.float16).astype(np.float32)
    assert check_planes(got, r16, d, plane_runs(d)) > 0
    check_points(got, r16, d, n_points=1000)
    check_windows(got, r16, d, window_points(d))


def test_fullsize_mover_windows(st, field, found):
    d, cube, _, _ = field
    got, _ = found
    # the bright movers are detected: the windows hold candidates
    assert check_windows(got, cube, d, window_points(d)) >= len(d["truth"]) // 2


def test_fullsize_normalisation(st, field):
    d, cube, mu, sd = field
    raw = torch.from_numpy(np.ascontiguousarray(d["frames"])).cuda()
    with st.Plan(d["field"], storage="f32", normalize=True, cr_clip=CR_CLIP) as p:
        gcube, gmu, gsd = p.normalize(0, raw)
    del raw
    assert np.all(np.abs(gsd - sd) <= 1e-12 * sd)
    assert np.all(np.abs(gmu - mu) <= 1e-12 * sd)
    g = gcube.cpu().numpy()
    del gcube
    torch.cuda.empty_cache()
    for i in range(0, g.shape[0], 16):  # frame blocks keep the temporaries small
        a, b = g[i:i + 16], cube[i:i + 16]
        tol = np.maximum(np.spacing(np.abs(b)), np.float32(1e-12))
        assert np.all(np.abs(a - b) <= tol), i


# ------------------------------------------------------------------ front end

FRONT_GROUP, FRONT_OVERLAP, FRONT_SUM = 50, 5, 13  # the benchmark's front-end configuration
N_PIX = 20000  # sampled pixels per median group


def test_fullsize_front_end(st, field):
    """Median removal over overlapping groups of 50 frames, sums of every 13
    frames and 2 x 2 binning of the raw 2048^2 x 256 cube: sums and binning
    compared whole, the medians on sampled pixels (the numpy oracle selects
    per pixel), all bit for bit."""
    from oracle import front
    from paper_2303_07293_gb300 import groups as grp
    d = field[0]
    fr = d["frames"]
    N, H, W = fr.shape
    frames = torch.from_numpy(np.ascontiguousarray(fr)).cuda()
    sums, ts = st.sum_frames(frames, d["times"], FRONT_SUM)
    osums, ots = front.sum_frames(fr, d["times"], FRONT_SUM)
    assert np.array_equal(sums.cpu().numpy(), osums, equal_nan=True)
    assert np.array_equal(ts, ots)
    del sums, osums
    binned = st.bin2x2(frames)
    assert np.array_equal(binned.cpu().numpy(), front.bin2x2(fr), equal_nan=True)
    del binned
    rng = np.random.default_rng(13)
    pix = np.sort(rng.choice(H * W, N_PIX, replace=False))
    pix_t = torch.from_numpy(pix).cuda()
    flat = fr.reshape(N, H * W)
    for s, e in grp.group_ranges(N, FRONT_GROUP, FRONT_OVERLAP):
        out, med = st.median_subtract(frames[s:e], with_median=True)
        got = out.reshape(e - s, H * W).index_select(1, pix_t).cpu().numpy()
        gmed = med.reshape(H * W).index_select(0, pix_t).cpu().numpy()
        ref, rmed = front.median_subtract(flat[s:e, pix][:, None, :])
        assert np.array_equal(gmed, rmed[0], equal_nan=True), (s, e)
        assert np.array_equal(got, ref[:, 0, :], equal_nan=True), (s, e)
        del out, med
    del frames
    torch.cuda.empty_cache()


# ------------------------------------------------------------------ refinement

REFINE_N = 4096     # candidates per call, as benchmarked
REFINE_SAMPLE = 128  # of them re-evaluated by the FP64 oracle
KINK_MARGIN = 1e-4   # > FP32 error of v dt (|v dt| <= 208 px: about 2.5e-5 px)


def refine_thetas(d, n, seed=9):
    """theta rows (vx, vy, x0, y0, F): the injected movers first, then random
    motions over the search grid's range and positions over the whole frame
    (cutouts hanging over the borders included); FP64 copies of the FP32
    values the GPU receives, and the integer cutout centres."""
    f = d["field"]
    rng = np.random.default_rng(seed)
    tr = np.asarray(d["truth"], np.float64)[:, [2, 3, 0, 1, 4]]
    m = min(len(tr), n)
    th = np.empty((n, 5))
    th[:m] = tr[:m]
    k = n - m
    th[m:, 0] = rng.uniform(f["vx0"], f["vx0"] + (f["nvx"] - 1) * f["dvx"], k)
    th[m:, 1] = rng.uniform(f["vy0"], f["vy0"] + (f["nvy"] - 1) * f["dvy"], k)
    th[m:, 2] = rng.uniform(0.0, f["width"] - 1.0, k)
    th[m:, 3] = rng.uniform(0.0, f["height"] - 1.0, k)
    th[m:, 4] = rng.uniform(0.5, 3.0, k)
    th = th.astype(np.float32).astype(np.float64)
    return th, np.rint(th[:, 2:4]).astype(np.int32)


def kink_free(th, dt, margin=KINK_MARGIN):
    """True where no frame's shift v dt (either axis) lies within margin of an
    integer, so the kernel (parameters rounded to FP32) and the oracle pick
    the same bilinear cell in every frame (the derivative in v jumps between
    cells); frames at dt = 0 shift by exactly 0 on both sides."""
    d = dt[dt != 0]
    ok = np.ones(len(th), bool)
    for ax in (0, 1):
        s = th[:, ax][:, None] * d[None, :]
        fr_ = s - np.floor(s)
        ok &= np.all((fr_ > margin) & (fr_ < 1.0 - margin), axis=1)
    return ok


def test_fullsize_refine_eval(st):
    """The refinement objective, S/N and adjoint of 4096 candidates on the
    2048^2 x 300-frame refinement field (the benchmark's batch and cutout),
    128 of them against the FP64 oracle with the small-size bars: J and S/N
    within 2e-4 relative, the gradient within 2e-4 of its largest component
    where no frame sits within 1e-4 px of a bilinear cell edge.  Shifts
    reach 208 px here (5 px in the small-size test); the kernel forms them
    in FP64 like the oracle, so the small-size bars hold unchanged."""
    d = synth.make_field("refine")
    cube = oracle.normalize(d["frames"], cr_clip=CR_CLIP)[0]
    del d["frames"]
    f = dict(d["field"], vx0=0.0, dvx=1.0, nvx=1, vy0=0.0, dvy=1.0, nvy=1)  # search: set-up only
    t, t_ref = d["times"], f["t_ref"]
    th, ce = refine_thetas(d, REFINE_N)
    frames = torch.from_numpy(cube).cuda()
    with st.Plan(f) as p:
        p.candidates(frames, t)
        J, snr, g = p.refine_eval(torch.tensor(th, dtype=torch.float32).cuda(), ce)
        J, snr, g = J.cpu().numpy(), snr.cpu().numpy(), g.cpu().numpy()
    del frames
    torch.cuda.empty_cache()
    assert np.all(np.isfinite(J)) and np.all(np.isfinite(snr)) and np.all(np.isfinite(g))
    rng = np.random.default_rng(17)
    idx = np.concatenate([np.arange(32), 32 + np.sort(rng.choice(REFINE_N - 32,
                                                                 REFINE_SAMPLE - 32,
                                                                 replace=False))])
    oJ, osnr, og = oracle.refine_eval(cube, t, t_ref, th[idx], ce[idx])
    assert np.all(np.abs(J[idx] - oJ) <= 2e-4 * (np.abs(oJ) + 1.0))
    assert np.all(np.abs(snr[idx] - osnr) <= 2e-4 * (np.abs(osnr) + 1.0))
    smooth = kink_free(th[idx], t - t_ref)
    assert smooth.sum() >= REFINE_SAMPLE // 2
    tol = 2e-4 * (np.abs(og).max(axis=1, keepdims=True) + 1.0)
    assert np.all((np.abs(g[idx] - og) <= tol)[smooth])


# ------------------------------------------------------------------ 1024^2 x 64 field

@pytest.fixture(scope="module")
def mid():
    d = synth.make_field("mid")
    cube = oracle.normalize(d["frames"], cr_clip=CR_CLIP)[0]
    return d, cube


def near_ties(cube, d, pts, mode="bilinear"):
    """For each (x, y, k): the smallest gap, in the FP64 stack, between S and
    its threshold or an in-frame neighbour's S, and the bar it is held to
    (2e-5 max(|S|, sqrt N), twice the value bar: both sides may err)."""
    f = d["field"]
    W, H, N = f["width"], f["height"], f["n_frames"]
    gaps, bars = [], []
    for x, y, k in pts:
        nb = [(x + dx, y + dy, k) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
              if 0 <= x + dx < W and 0 <= y + dy < H]
        S64, C64 = oracle.stack_points(cube, d["times"], f, np.array(nb, np.int32), mode=mode)
        c = nb.index((x, y, k))
        thr = float(np.float32(f["snr_threshold"] * np.sqrt(C64[c])))
        gaps.append(min([abs(S64[c] - thr)] +
                        [abs(S64[c] - S64[j]) for j in range(len(nb)) if j != c]))
        bars.append(2e-5 * max(abs(S64[c]), np.sqrt(N)))
    return np.array(gaps), np.array(bars)


def check_bilinear(got, cube, d, ref, region):
    """Bilinear candidates against the FP64 oracle's list ref over a region
    (a boolean over got): common candidates within 1e-5 max(|S64|, sqrt N)
    with the same coverage, every candidate of only one list a near-tie."""
    N = d["field"]["n_frames"]
    sel = got[region]
    gk = _key(sel["x"], sel["y"], sel["k"])
    rk = _key(ref["x"], ref["y"], ref["k"])
    both_g, both_r = np.isin(gk, rk), np.isin(rk, gk)
    assert np.array_equal(sel["n_cov"][both_g], ref["n_cov"][both_r])
    s64 = ref["stack"][both_r]
    assert np.all(np.abs(sel["stack"][both_g] - s64) <= 1e-5 * np.maximum(np.abs(s64), np.sqrt(N)))
    only = [(int(r["x"]), int(r["y"]), int(r["k"])) for r in sel[~both_g]] + \
           [(int(r["x"]), int(r["y"]), int(r["k"])) for r in ref[~both_r]]
    if only:
        gaps, bars = near_ties(cube, d, only)
        assert np.all(gaps <= bars), [p for p, g_, b_ in zip(only, gaps, bars) if g_ > b_]
    return int(both_g.sum()), len(only)


@pytest.mark.parametrize("mode,storage", [("nearest", "f32"), ("bilinear", "f32"),
                                          ("nearest", "f16"), ("nearest", "bf16")])
def test_fullsize_mid(st, mid, mode, storage):
    """The 1024^2 x 64-frame field (2 h, star blobs masked, 20 movers) with the
    161 x 161 grid (+-40 px/h, step 0.5), in the benchmark's configuration,
    for nearest shifts (bit-exact: whole plane runs, sampled candidates,
    mover windows; FP16 / BF16 storage against the oracle on the frames
    rounded to the storage type) and bilinear shifts (against the FP64
    oracle: plane runs and mover windows with the bilinear bars, sampled
    candidates' values)."""
    d, cube32 = mid
    f = d["field"]
    cube = {"f32": lambda c: c, "f16": lambda c: c.astype(np.float16).astype(np.float32),
            "bf16": oracle.round_bf16}[storage](cube32)
    frames = torch.from_numpy(cube32).cuda()
    with st.Plan(f, storage=storage, mode=mode, tile=-1, pending_capacity=1 << 24) as p:
        got = p.candidates(frames, d["times"], capacity=1 << 22)
        assert p.last_stack_variant(0) == 1, "the register-window kernel must run"
    del frames
    torch.cuda.empty_cache()
    assert len(got) > 0 and np.all(np.diff(_key(got["x"], got["y"], got["k"])) > 0)
    starts = plane_runs(d)
    if mode == "nearest":
        assert check_planes(got, cube, d, starts) > 0
        check_points(got, cube, d)
        assert check_windows(got, cube, d, window_points(d)) > 0
        return
    common = 0
    for k0 in starts:
        ref = oracle.search(cube, d["times"], f, mode="bilinear", prec="fp64", k_begin=k0,
                            k_end=k0 + RUN)
        common += check_bilinear(got, cube, d, ref, (got["k"] >= k0) & (got["k"] < k0 + RUN))[0]
    assert common > 0
    pts = window_points(d)
    ok, S, Cv, snr = oracle.candidates_at(cube, d["times"], f, pts, mode="bilinear",
                                          prec="fp64")
    want = pts[ok]
    ref = np.zeros(len(want), dtype=[("x", np.int32), ("y", np.int32), ("k", np.int32),
                                      ("n_cov", np.int32), ("stack", np.float64)])
    ref["x"], ref["y"], ref["k"] = want[:, 0], want[:, 1], want[:, 2]
    ref["n_cov"], ref["stack"] = Cv[ok], S[ok]
    region = np.isin(_key(got["x"], got["y"], got["k"]), _key(pts[:, 0], pts[:, 1], pts[:, 2]))
    check_bilinear(got, cube, d, ref, region)
    rng = np.random.default_rng(5)
    c = got[np.sort(rng.choice(len(got), min(N_POINTS, len(got)), replace=False))]
    S64, C64 = oracle.stack_points(cube, d["times"], f,
                                   np.stack([c["x"], c["y"], c["k"]], axis=1), mode="bilinear")
    assert np.array_equal(c["n_cov"], C64)
    assert np.all(np.abs(c["stack"] - S64) <=
                  1e-5 * np.maximum(np.abs(S64), np.sqrt(f["n_frames"])))


# ------------------------------------------------------------------ batched fields

BATCH_FIELDS = (23, 5, 15, 14)  # of the 24-field batch: 512^2-2048^2, 45-289 frames


@pytest.fixture(scope="module")
def batch():
    base = synth.BASE_SEED + 4
    ds = [synth.make_field("batched", seed=base, index=j) for j in BATCH_FIELDS]
    cubes = [oracle.normalize(d["frames"], cr_clip=CR_CLIP)[0] for d in ds]
    for d in ds:
        del d["frames"]
    return ds, cubes


def test_fullsize_batched_fields_one_launch(st, batch):
    """Four fields of the batched workload at their full sizes in one plan, in
    the benchmark's configuration of the batch: FP16 storage, autotuned
    variant, the device part captured in a CUDA graph and replayed, one
    persistent launch over all fields.  Against the oracle on each field's
    frames rounded to FP16 (the same FP32 adds, bit for bit): plane runs,
    sampled candidates and mover windows of every field."""
    ds, cubes = batch
    frames = [torch.from_numpy(c).cuda() for c in cubes]
    times = [d["times"] for d in ds]
    with st.Plan([d["field"] for d in ds], storage="f16", mode="nearest", tile=-1,
                 use_graph=True, pending_capacity=1 << 24) as p:
        first = p.candidates(frames, times, capacity=1 << 22)
        got = p.candidates(frames, times, capacity=1 << 22)
        assert p.last_graph_replayed()
        assert [p.last_stack_variant(i) for i in range(len(ds))] == [1] * len(ds)
        _, stack_launches = p.last_stack_kernel_time()
    del frames
    torch.cuda.empty_cache()
    assert stack_launches == 1
    assert got.tobytes() == first.tobytes()
    assert np.all(np.diff(got["field"]) >= 0)
    for j, (d, c) in enumerate(zip(ds, cubes)):
        r16 = c.astype(np.float16).astype(np.float32)
        g = got[got["field"] == j]
        assert len(g) > 0
        assert np.all(np.diff(_key(g["x"], g["y"], g["k"])) > 0)
        assert check_planes(g, r16, d, plane_runs(d)) >= 0
        check_points(g, r16, d, n_points=500)
        check_windows(g, r16, d, window_points(d))


# ------------------------------------------------------------------ multi-night stack

def test_fullsize_multinight(st):
    """The multi-night workload at its full size (two nights of 64 frames of
    1024^2 px 24 h apart, a grid of 1 px over the whole baseline), searched as
    benchmarked (FP32, autotuned register-window variant): plane runs,
    sampled candidates and mover windows bit for bit with the oracle."""
    d = synth.make_field("multinight")
    cube = oracle.normalize(d["frames"], cr_clip=CR_CLIP)[0]
    del d["frames"]
    frames = torch.from_numpy(cube).cuda()
    with st.Plan(d["field"], storage="f32", mode="nearest", tile=-1,
                 pending_capacity=1 << 24) as p:
        got = p.candidates(frames, d["times"], capacity=1 << 22)
        assert p.last_stack_variant(0) == 1
    del frames
    torch.cuda.empty_cache()
    assert len(got) > 0 and np.all(np.diff(_key(got["x"], got["y"], got["k"])) > 0)
    assert check_planes(got, cube, d, plane_runs(d)) >= 0
    check_points(got, cube, d, n_points=1000)
    check_windows(got, cube, d, window_points(d))
