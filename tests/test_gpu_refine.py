"""GPU parity of the refinement (forward + hand-written adjoint) against the
FP64 oracle of oracle/refine_oracle.c, the autograd binding, and the Adam
refinement of an injected mover (not in the paper: a continuous refinement of
the grid detections of Sec. 2.1)."""
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


def make(seed=41, N=24, W=160, H=150, mover=(80.3, 74.6, 0.45, -0.3, 2.5)):
    fr = synth.noise(N, H, W, seed=seed)
    t = np.arange(N, dtype=np.float64) * 0.5
    t_ref = float(t[N // 2])
    synth.render_movers(fr, t, t_ref, [list(mover)], fwhm=3.0)
    f = synth.field_params(W, H, N, t_ref, -1.0, 0.25, 9, -1.0, 0.25, 9, tau=4.0)
    return fr, t, f


def kink_free(v, dt, margin=0.02):
    # frames with dt = 0 sample exact integers in FP32 and FP64 alike
    d = dt[dt != 0]
    fr_ = v * d - np.floor(v * d)
    return bool(np.all((fr_ > margin) & (fr_ < 1 - margin)))


def test_refine_eval_matches_oracle(st):
    fr, t, f = make()
    rng = np.random.default_rng(3)
    th, ce = [], []
    dt = t - f["t_ref"]
    for _ in range(100000):
        if len(th) == 24:
            break
        vx, vy = rng.uniform(-0.9, 0.9, 2)
        if not (kink_free(vx, dt) and kink_free(vy, dt)):
            continue
        x0, y0 = rng.uniform(40, 120, 2)
        th.append([vx, vy, x0, y0, rng.uniform(0.5, 3.0)])
        ce.append([int(round(x0)), int(round(y0))])
    assert len(th) == 24
    th = np.array(th)
    ce = np.array(ce, np.int32)
    with st.Plan(f, mode="nearest") as p:
        p.candidates(torch.from_numpy(fr).cuda(), t)
        J, snr, g = p.refine_eval(torch.tensor(th, dtype=torch.float32).cuda(), ce)
    oJ, osnr, og = oracle.refine_eval(fr, t, f["t_ref"], th.astype(np.float32).astype(np.float64),
                                      ce)
    J, snr, g = J.cpu().numpy(), snr.cpu().numpy(), g.cpu().numpy()
    # FP32 sums of N x 4096 terms against FP64: relative 2e-4 of the scale
    scale = np.abs(og).max(axis=1, keepdims=True) + 1.0
    assert np.all(np.abs(J - oJ) <= 2e-4 * (np.abs(oJ) + 1.0))
    assert np.all(np.abs(snr - osnr) <= 2e-4 * (np.abs(osnr) + 1.0))
    assert np.all(np.abs(g - og) <= 2e-4 * scale), np.abs(g - og).max()


def test_refine_eval_edges_and_interior(st):
    # cutouts hanging over each border and corner (zero taps outside) and
    # cutouts whose every frame footprint is inside (the unchecked-load path)
    fr, t, f = make(seed=45, W=256, H=200)
    rng = np.random.default_rng(5)
    dt = t - f["t_ref"]
    cen = [(3, 100), (252, 100), (128, 2), (128, 198), (0, 0), (255, 199), (128, 100),
           (100, 90), (150, 110)]
    th, ce = [], []
    for cx, cy in cen:
        while True:
            vx, vy = rng.uniform(-0.9, 0.9, 2)
            if kink_free(vx, dt) and kink_free(vy, dt):
                break
        th.append([vx, vy, cx + rng.uniform(-0.5, 0.5), cy + rng.uniform(-0.5, 0.5), 1.5])
        ce.append([cx, cy])
    th = np.array(th)
    ce = np.array(ce, np.int32)
    with st.Plan(f) as p:
        p.candidates(torch.from_numpy(fr).cuda(), t)
        J, snr, g = p.refine_eval(torch.tensor(th, dtype=torch.float32).cuda(), ce)
    oJ, osnr, og = oracle.refine_eval(fr, t, f["t_ref"], th.astype(np.float32).astype(np.float64),
                                      ce)
    J, snr, g = J.cpu().numpy(), snr.cpu().numpy(), g.cpu().numpy()
    scale = np.abs(og).max(axis=1, keepdims=True) + 1.0
    assert np.all(np.abs(J - oJ) <= 2e-4 * (np.abs(oJ) + 1.0))
    assert np.all(np.abs(snr - osnr) <= 2e-4 * (np.abs(osnr) + 1.0))
    assert np.all(np.abs(g - og) <= 2e-4 * scale), np.abs(g - og).max()


def test_autograd_backward_is_the_adjoint(st):
    fr, t, f = make(seed=43)
    th = torch.tensor([[0.37, -0.23, 80.4, 74.3, 2.2]], dtype=torch.float32, device="cuda",
                      requires_grad=True)
    ce = torch.tensor([[80, 74]], dtype=torch.int32, device="cuda")
    with st.Plan(f) as p:
        p.candidates(torch.from_numpy(fr).cuda(), t)
        J = st.refine_objective(th, p, ce)
        (2.0 * J.sum()).backward()
        _, _, g = p.refine_eval(th.detach(), ce)
    assert torch.allclose(th.grad, 2.0 * g, rtol=0, atol=0)
    og = oracle.refine_eval(fr, t, f["t_ref"], th.detach().cpu().double().numpy(), [[80, 74]])[2]
    assert np.all(np.abs(th.grad.cpu().numpy() / 2.0 - og) <= 2e-4 * (np.abs(og).max() + 1.0))


def test_adam_refinement_recovers_injected_motion(st):
    truth = (80.3, 74.6, 0.45, -0.3, 2.5)
    fr, t, f = make(seed=47, mover=truth)
    dev_fr = torch.from_numpy(fr).cuda()
    with st.Plan(f) as p:
        out, n, status = p.search(dev_fr, t, capacity=1 << 16)
        c = p.to_numpy(out, n)
        # the brightest grid detection of the mover
        best = int(np.argmax(c["stack"]))
        rec = p.refine(out[best:best + 1], n=1, steps=150, lr_pos=0.02, lr_vel=0.005)
    r = rec[0]
    # the refined point is at least as likely as the injected truth under the
    # FP64 oracle (each with F at its optimum) and within statistical error
    def j_at(vx, vy, x0, y0):
        _, snr, _ = oracle.refine_eval(fr, t, f["t_ref"], [[vx, vy, x0, y0, 1.0]],
                                       [[int(c["x"][best]), int(c["y"][best])]], 3.0, grad=False)
        return snr[0] ** 2 / 2  # J at F_hat
    j_ref = j_at(r["vx"], r["vy"], r["x0"], r["y0"])
    j_true = j_at(truth[2], truth[3], truth[0], truth[1])
    assert j_ref >= j_true * (1 - 1e-4), (j_ref, j_true)
    assert abs(r["x0"] - truth[0]) < 0.2 and abs(r["y0"] - truth[1]) < 0.2, r
    assert abs(r["vx"] - truth[2]) < 0.1 and abs(r["vy"] - truth[3]) < 0.1, r
    assert abs(r["flux"] - truth[4]) < 0.15 * truth[4], r
    assert r["snr"] > 10


def _noiseless(t, t_ref, truth, W=160, H=150):
    fr = np.zeros((len(t), H, W), np.float32)
    x0, y0, vx, vy, A = truth
    synth.render_movers(fr, t, t_ref, [[x0, y0, vx, vy, A]], fwhm=3.0)
    return fr


def _gn_field(t, t_ref, vx0, dvx, vy0, dvy, W=160, H=150):
    return synth.field_params(W, H, len(t), t_ref, vx0, dvx, 3, vy0, dvy, 3, tau=3.0)


def _one_candidate(p, x, y, k):
    # a search record as the refinement reads it: pixel, grid index, field 0
    rec = np.zeros(7, np.int32)
    rec[0], rec[1], rec[2], rec[3] = x, y, k, 0
    return torch.from_numpy(rec[None]).cuda()


def test_gauss_newton_steps_equal_the_oracle(st):
    # Gauss-Newton (optimizer 1) from a grid candidate next to a noiseless
    # mover: after each of 1..6 steps the GPU's (vx, vy, x0, y0) equal the
    # FP64 oracle's steps (refine_gn_step, damping 1) from the same start.
    # The GPU forms the step from FP32 sums of N x 4096 terms (relative
    # 2e-4, the eval bar); a step's solution carries that error times the
    # system's condition (a few here), so each parameter is held to 2e-3 of
    # the oracle's move so far plus 2e-4 px (position) / 2e-5 px per time
    # unit (motion).
    t = np.array([0.0, 0.7, 1.6, 2.1, 2.9, 3.3, 4.8, 5.2, 6.5, 7.9, 8.4])
    t_ref = 2.1
    truth = np.array([70.3, 58.6, 1.37, -0.83, 2.0])      # x0, y0, vx, vy, A
    fr = _noiseless(t, t_ref, truth)
    # grid velocity (1.31, 0.77): 0.06 off the truth; pixel (70, 59).  This
    # start keeps every frame's shift at least 2.5e-3 px from a bilinear cell
    # edge along the whole trajectory (checked below), where the objective's
    # slopes jump and FP32 and FP64 parameters could take different cells
    f = _gn_field(t, t_ref, 1.19, 0.12, -0.89, 0.12)
    k = 1 * 3 + 1
    start = np.array([[np.float32(1.19 + 0.12), np.float32(-0.89 + 0.12), 70.0, 59.0, 1.0]])
    dtn = (t - t_ref)[t != t_ref]
    dev_fr = torch.from_numpy(fr).cuda()
    th = start.astype(np.float64)
    with st.Plan(f) as p:
        p.candidates(dev_fr, t)
        for steps in range(1, 7):
            rec = p.refine(_one_candidate(p, 70, 59, k), n=1, steps=steps, optimizer="gn",
                           damping=1.0)[0]
            th_prev = th.copy()
            for v in th_prev[0, :2]:
                assert np.abs(v * dtn - np.round(v * dtn)).min() > 1e-3
            th = oracle.refine_gn_step(fr, t, t_ref, th, [[70, 59]], damping=1.0)
            got = np.array([rec["vx"], rec["vy"], rec["x0"], rec["y0"]], np.float64)
            moved = np.abs(th[0, :4] - start[0, :4])
            bar = 2e-3 * moved + np.array([2e-5, 2e-5, 2e-4, 2e-4])
            assert np.all(np.abs(got - th[0, :4]) <= bar), (steps, got, th[0, :4], th_prev)
    # within 0.05 of the truth (the oracle's pin); the flux within 10 %
    # (bilinear resampling of the rendered PSF lowers the matched-filter flux
    # by about 4 % at the oracle's own end point)
    err = np.abs(np.array([rec["x0"], rec["y0"], rec["vx"], rec["vy"]]) - truth[:4])
    assert err.max() <= 0.05, err
    assert abs(rec["flux"] - truth[4]) <= 0.1 * truth[4]


def test_gauss_newton_refinement_of_a_noisy_mover(st):
    # the injected mover of the Adam test: 20 damped Gauss-Newton steps end
    # at least as likely as the truth under the FP64 oracle and within the
    # same error as Adam's 150 steps
    truth = (80.3, 74.6, 0.45, -0.3, 2.5)
    fr, t, f = make(seed=47, mover=truth)
    dev_fr = torch.from_numpy(fr).cuda()
    with st.Plan(f) as p:
        out, n, status = p.search(dev_fr, t, capacity=1 << 16)
        c = p.to_numpy(out, n)
        best = int(np.argmax(c["stack"]))
        r = p.refine(out[best:best + 1], n=1, steps=20, optimizer="gn", damping=1.0)[0]
        with pytest.raises(st.StError):
            p.refine(out[best:best + 1], n=1, steps=2, optimizer="gn", damping=-1.0)

    def j_at(vx, vy, x0, y0):
        _, snr, _ = oracle.refine_eval(fr, t, f["t_ref"], [[vx, vy, x0, y0, 1.0]],
                                       [[int(c["x"][best]), int(c["y"][best])]], 3.0, grad=False)
        return snr[0] ** 2 / 2
    assert j_at(r["vx"], r["vy"], r["x0"], r["y0"]) >= \
        j_at(truth[2], truth[3], truth[0], truth[1]) * (1 - 1e-4)
    assert abs(r["x0"] - truth[0]) < 0.2 and abs(r["y0"] - truth[1]) < 0.2, r
    assert abs(r["vx"] - truth[2]) < 0.1 and abs(r["vy"] - truth[3]) < 0.1, r
    assert abs(r["flux"] - truth[4]) < 0.15 * truth[4], r
