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
