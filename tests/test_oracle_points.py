"""The point-wise detection rule of the oracle (``oracle.candidates_at``,
used where a field is too large to search whole) against the oracle's whole
search (``oracle.search``, itself pinned by the hand-built rule fixtures):
at every pixel of the checked velocity planes, a point is a candidate of one
exactly when it is a candidate of the other, with the same stack, coverage
and S/N; nearest and bilinear shifts, FP32-sequential and FP64 sums, a
lowered threshold (dense candidates, plateaus of equal values) and edge
coverage."""
import numpy as np
import pytest

import oracle
import synth


def _cases():
    d = synth.make_field("tiny")
    yield "tiny", d["frames"], d["times"], d["field"]
    fr = synth.noise(13, 53, 77, seed=3)
    rng = np.random.default_rng(3)
    t = np.sort(rng.uniform(0.0, 3.0, 13))
    f = synth.field_params(77, 53, 13, float(t[6]), -2.1, 0.55, 9, -1.3, 0.45, 7, tau=2.0)
    synth.render_movers(fr, t, f["t_ref"], [[30.0, 20.0, 1.1, -0.8, 2.5]])
    yield "ragged", fr, t, f
    q = np.round(synth.noise(9, 24, 31, seed=4) * 2.0).astype(np.float32)  # many equal sums
    tq = np.arange(9, dtype=np.float64)
    fq = synth.field_params(31, 24, 9, 4.0, -2.0, 1.0, 5, -2.0, 1.0, 5, tau=1.0)
    yield "plateaus", q, tq, fq


@pytest.mark.parametrize("mode,prec", [("nearest", "fp32"), ("nearest", "fp64"),
                                       ("bilinear", "fp32"), ("bilinear", "fp64")])
def test_point_rule_equals_whole_search(mode, prec):
    checked = 0
    for name, fr, t, f in _cases():
        fr = np.nan_to_num(fr, nan=0.0)
        nk = f["nvx"] * f["nvy"]
        ks = sorted({0, nk // 3, nk // 2, nk - 1})
        H, W = f["height"], f["width"]
        for k in ks:
            ref = oracle.search(fr, t, f, mode=mode, prec=prec, k_begin=k, k_end=k + 1)
            yy, xx = np.mgrid[0:H, 0:W]
            xyk = np.stack([xx.ravel(), yy.ravel(), np.full(H * W, k)], axis=1)
            ok, S, Cv, snr = oracle.candidates_at(fr, t, f, xyk, mode=mode, prec=prec)
            sel = np.flatnonzero(ok)                       # raster order = search order
            assert np.array_equal(xyk[sel, 0], ref["x"]), (name, k)
            assert np.array_equal(xyk[sel, 1], ref["y"]), (name, k)
            assert np.array_equal(Cv[sel], ref["n_cov"]), (name, k)
            assert np.array_equal(S[sel], ref["stack"]), (name, k)
            assert np.array_equal(snr[sel], ref["snr"]), (name, k)
            checked += len(sel)
    assert checked > 50
