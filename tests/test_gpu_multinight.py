"""Multi-night stacks (next row 4): frames of two nights 24 h apart, a grid
whose step is 1 px over the whole baseline (a large grid for slow movers).
The register-window kernel must handle the sparse time sampling: stack
values, coverage and candidates bit-exact with the FP32-sequential oracle,
and the injected slow movers recovered."""
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


@pytest.mark.parametrize("nights,tile", [(2, 0), (3, 0), (2, 3)])
def test_multinight_bitexact_and_recovery(st, nights, tile):
    d = synth.make_field("multinight", width=128, n_frames=12 * nights, nights=nights,
                         vmax=1.0, n_movers=2, tau=4.0)
    fr, t, f = d["frames"], d["times"], d["field"]
    ks = np.arange(f["nvx"] * f["nvy"], dtype=np.int32)[::7]
    with st.Plan(f, tile=tile) as p:
        got = p.candidates(torch.from_numpy(fr).cuda(), t)
        assert p.last_stack_variant(0) == 1, "register-window kernel not used"
        S, Cv = p.dump_stack(0, torch.from_numpy(fr).cuda(), t, np.arange(f["nvx"] * f["nvy"],
                                                                            dtype=np.int32))
    ref = oracle.search(fr, t, f, prec="fp32")
    assert got[["x", "y", "k", "n_cov"]].tolist() == ref[["x", "y", "k", "n_cov"]].tolist()
    assert np.array_equal(got["stack"], ref["stack"].astype(np.float32))
    oS, oC = oracle.stack_planes(fr, t, f, ks, prec="fp32")
    assert np.array_equal(S.cpu().numpy()[ks], oS.astype(np.float32))
    assert np.array_equal(Cv.cpu().numpy()[ks], oC)
    for m in d["truth"]:
        a, b, _ = synth.velocity_index(f, m[2], m[3])
        hit = (np.abs(got["x"] - m[0]) <= 2) & (np.abs(got["y"] - m[1]) <= 2) & \
              (np.abs(got["k"] % f["nvx"] - a) <= 1) & (np.abs(got["k"] // f["nvx"] - b) <= 1)
        assert hit.any(), m
