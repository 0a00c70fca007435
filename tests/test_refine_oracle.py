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
