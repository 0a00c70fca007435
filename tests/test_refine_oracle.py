"""Pins of the FP64 refinement oracle (CPU only).

The refinement maximises a Gaussian matched-filter log-likelihood of the
bilinear stack on a 64 x 64 cutout (oracle/refine_oracle.c states the
definitions).  Pinned by: closed forms for a noiseless mover rendered with the
template's PSF (F_hat = A, J = N A^2 <g,g> / 2, zero position gradient at the
truth), a linear ramp (exact velocity derivative), and central finite
differences at a point clear of bilinear kinks.
"""
import math

import numpy as np

import oracle
import synth

FWHM = 3.0
SIG = FWHM / (2 * math.sqrt(2 * math.log(2)))


def gauss_grid(cx, cy, x0, y0):
    u = np.arange(64) + cx - 32
    w = np.arange(64) + cy - 32
    X, Y = np.meshgrid(u, w)
    return np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / (2 * SIG ** 2)), X, Y


def test_noiseless_mover_closed_form():
    N, H, W = 9, 120, 140
    t = np.arange(N, dtype=np.float64)
    t_ref = 4.0
    x0, y0, vx, vy, A = 70, 58, 2, -1, 1.7
    fr = np.zeros((N, H, W), np.float32)
    synth.render_movers(fr, t, t_ref, [[x0, y0, vx, vy, A]], fwhm=FWHM)
    g, _, _ = gauss_grid(x0, y0, x0, y0)
    gg = float((g * g).sum())
    J, snr, grad = oracle.refine_eval(fr, t, t_ref, [[vx, vy, x0, y0, A]], [[x0, y0]], FWHM)
    # the rendered PSF is cut at 4 sigma; the template is not: relative 1e-7
    assert abs(J[0] - 0.5 * N * A * A * gg) <= 1e-6 * J[0]
    assert abs(snr[0] - A * math.sqrt(N * gg)) <= 1e-6 * snr[0]
    assert abs(grad[0, 2]) < 1e-6 and abs(grad[0, 3]) < 1e-6   # position
    assert abs(grad[0, 4]) < 1e-6 * N * gg                     # F at its optimum
    # F_hat = <g,S>/(N<g,g>) = A: dJ/dF vanishes there and is linear in F
    J2, _, grad2 = oracle.refine_eval(fr, t, t_ref, [[vx, vy, x0, y0, 2 * A]], [[x0, y0]], FWHM)
    assert abs(grad2[0, 4] - (-A * N * gg)) <= 1e-6 * A * N * gg


def test_linear_ramp_velocity_derivative():
    # I = alpha x + beta y + gamma in every frame: S is linear in the motion
    # and dJ/dvx = F alpha (sum_i dt_i) (sum_p g)
    N, H, W = 7, 160, 160
    t = np.array([0.0, 0.4, 1.3, 1.9, 2.2, 3.7, 4.1])
    t_ref = 1.9
    al, be, ga = 0.25, -0.5, 3.0
    yy, xx = np.mgrid[0:H, 0:W]
    fr = np.broadcast_to((al * xx + be * yy + ga).astype(np.float32), (N, H, W)).copy()
    th = [0.61, -0.37, 80.3, 79.6, 1.3]
    J, snr, grad = oracle.refine_eval(fr, t, t_ref, [th], [[80, 80]], FWHM)
    g, X, Y = gauss_grid(80, 80, th[2], th[3])
    sdt = float((t - t_ref).sum())
    assert abs(grad[0, 0] - th[4] * al * sdt * g.sum()) < 1e-9 * abs(th[4] * g.sum())
    assert abs(grad[0, 1] - th[4] * be * sdt * g.sum()) < 1e-9 * abs(th[4] * g.sum())
    # and S itself: <g, S> with S(p) = sum_i (al (x + vx dt) + be (y + vy dt) + ga)
    dt = t - t_ref
    S = sum(al * (X + th[0] * d) + be * (Y + th[1] * d) + ga for d in dt)
    gS = float((g * S).sum())
    assert abs(J[0] - (th[4] * gS - 0.5 * th[4] ** 2 * N * (g * g).sum())) < 1e-8 * abs(J[0])


def test_gradient_matches_central_differences():
    N, H, W = 8, 110, 110
    t = np.arange(N, dtype=np.float64)
    t_ref = 3.5
    fr = synth.noise(N, H, W, seed=31)
    synth.render_movers(fr, t, t_ref, [[55.2, 54.6, 0.4, -0.25, 3.0]], fwhm=FWHM)
    # fractions of vx dt and vy dt stay in [0.07, 0.93] for every frame, so a
    # step of 1e-3 px/unit never crosses a bilinear kink
    th = np.array([0.37, -0.23, 55.4, 54.3, 2.6])
    for v, dt in ((th[0], t - t_ref), (th[1], t - t_ref)):
        fr_ = (v * dt) - np.floor(v * dt)
        assert np.all((fr_ > 0.05) & (fr_ < 0.95))
    J, _, grad = oracle.refine_eval(fr, t, t_ref, [th], [[55, 55]], FWHM)
    for k in range(5):
        h = 1e-3
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        Jp, _, _ = oracle.refine_eval(fr, t, t_ref, [tp], [[55, 55]], FWHM, grad=False)
        Jm, _, _ = oracle.refine_eval(fr, t, t_ref, [tm], [[55, 55]], FWHM, grad=False)
        fd = (Jp[0] - Jm[0]) / (2 * h)
        assert abs(fd - grad[0, k]) <= 1e-5 * max(1.0, abs(grad[0, k])), (k, fd, grad[0, k])


# ------------------------------------------------ Gauss-Newton curvature (optimizer 1)

def _noiseless(t, t_ref, theta, H=120, W=140):
    """Frames of one mover with parameters theta = (vx, vy, x0, y0, A)."""
    vx, vy, x0, y0, A = theta
    fr = np.zeros((len(t), H, W), np.float32)
    synth.render_movers(fr, t, t_ref, [[x0, y0, vx, vy, A]], fwhm=FWHM)
    return fr


def test_gauss_newton_curvature_is_the_hessian_of_a_noiseless_fit():
    # zero residuals (a mover rendered with the template's PSF on integer
    # shifts, at its true parameters): J^T J equals -Hessian(J) exactly in
    # position and flux, where J is smooth; central differences of the
    # analytic gradient give that Hessian
    t = np.arange(9, dtype=np.float64)
    t_ref = 3.0                                    # sum of dt != 0: couplings present
    truth = (2.0, -1.0, 70.0, 58.0, 1.7)
    fr = _noiseless(t, t_ref, truth)
    th = np.array([truth])
    ce = [[70, 58]]
    Hm = oracle.refine_gn_matrix(t, t_ref, th, ce)[0]
    assert np.allclose(Hm, Hm.T)
    h = 1e-4
    for a in (2, 3, 4):
        tp, tm = th.copy(), th.copy()
        tp[0, a] += h
        tm[0, a] -= h
        col = (oracle.refine_eval(fr, t, t_ref, tp, ce)[2][0] -
               oracle.refine_eval(fr, t, t_ref, tm, ce)[2][0]) / (2 * h)
        for b in (2, 3, 4):
            assert abs(col[b] + Hm[b, a]) <= 1e-5 * abs(Hm[4, 4]), (a, b)
    # closed forms of the isotropic template, <Gx,Gx> = pi/2 and <g,g> =
    # pi s^2 (integrals; the cutout sums them on the pixel grid, where a
    # Gaussian of width s/sqrt 2 = 0.9 px aliases below 1e-4)
    N = len(t)
    assert abs(Hm[2, 2] - 1.7 ** 2 * N * math.pi / 2) <= 1e-4 * Hm[2, 2]
    assert abs(Hm[4, 4] - N * math.pi * SIG ** 2) <= 1e-4 * Hm[4, 4]
    T1, T2 = float((t - t_ref).sum()), float(((t - t_ref) ** 2).sum())
    assert abs(Hm[0, 0] - T2 / N * Hm[2, 2]) <= 1e-9 * Hm[0, 0]
    assert abs(Hm[0, 2] - T1 / N * Hm[2, 2]) <= 1e-9 * abs(Hm[0, 2])


def test_gauss_newton_motion_position_coupling():
    # d/dvx (dJ/dx0) of the bilinear stack approaches -[vx, x0] of J^T J;
    # the bilinear cell slopes of a sampled PSF (FWHM 3 px) stand in for its
    # derivative, within 15 %
    t = np.array([0.0, 0.7, 1.6, 2.1, 2.9, 3.3, 4.8, 5.2, 6.5, 7.9, 8.4])
    t_ref = 2.1
    truth = (1.37, -0.83, 70.3, 58.6, 2.0)
    fr = _noiseless(t, t_ref, truth)
    th = np.array([truth])
    ce = [[70, 59]]
    Hm = oracle.refine_gn_matrix(t, t_ref, th, ce)[0]
    h = 1e-3
    for a, b in ((0, 2), (1, 3)):
        tp, tm = th.copy(), th.copy()
        tp[0, a] += h
        tm[0, a] -= h
        d = (oracle.refine_eval(fr, t, t_ref, tp, ce)[2][0][b] -
             oracle.refine_eval(fr, t, t_ref, tm, ce)[2][0][b]) / (2 * h)
        assert abs(d + Hm[a, b]) <= 0.15 * abs(Hm[a, b]), (a, b, d, Hm[a, b])


def test_gauss_newton_steps_approach_the_truth():
    # damped steps from 0.4 px (and the matching motion) off a noiseless
    # mover settle within 0.05 of the truth in every parameter; the bilinear
    # objective's own maximum lies about 0.01 from it
    t = np.array([0.0, 0.7, 1.6, 2.1, 2.9, 3.3, 4.8, 5.2, 6.5, 7.9, 8.4])
    t_ref = 2.1
    truth = np.array([1.37, -0.83, 70.3, 58.6, 2.0])
    fr = _noiseless(t, t_ref, truth)
    ce = [[70, 59]]
    th = truth[None].copy()
    th[0, :4] += [0.4 / 6.3, -0.3 / 6.3, 0.4, -0.3]
    errs = []
    for _ in range(6):
        errs.append(np.abs(th[0, :4] - truth[:4]).max())
        th = oracle.refine_gn_step(fr, t, t_ref, th, ce, damping=1.0)
    errs.append(np.abs(th[0, :4] - truth[:4]).max())
    assert errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1]
    assert errs[-1] <= 0.05
