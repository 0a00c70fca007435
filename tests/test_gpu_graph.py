"""CUDA-graph capture of the search (use_graph, row a8).

The device part of a search (normalisation, the stack launches, the
local-maximum resolver and the counter read-back) is captured on the first
search with given frame pointers and timestamps and replayed afterwards.  A
replay must give exactly the candidates of a plan without graphs, also after
the frames' contents change in place, after the timestamps change (tables are
rebuilt and the graph is captured again) and after the frame pointers change.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def fields(n=3, seed=60):
    out = []
    for j in range(n):
        d = synth.make_field("mid", seed=seed + j, width=96 + 32 * j, n_frames=12 + 7 * j,
                             nv=9 + 2 * j, n_movers=3, n_blobs=4)
        out.append(d)
    return out


@pytest.mark.parametrize("storage,mode", [("f32", "nearest"), ("f16", "nearest"),
                                          ("f32", "bilinear")])
def test_graph_replay_equals_direct(st, storage, mode):
    ds = fields()
    fs = [d["field"] for d in ds]
    ts = [d["times"] for d in ds]
    frames = [dev(d["frames"] * 2.0 + 7.0) for d in ds]
    kw = dict(storage=storage, mode=mode, normalize=True)
    with st.Plan(fs, **kw) as p0:
        out0, n0, s0 = p0.search(frames, ts, capacity=1 << 16)
        ref = p0.to_numpy(out0, n0)
        assert not p0.last_graph_replayed()
    with st.Plan(fs, use_graph=True, **kw) as p:
        for rep in range(3):
            out, n, s = p.search(frames, ts, capacity=1 << 16)
            assert s == st.ST_OK and p.last_graph_replayed(), (rep, st.lib().st_last_error())
            assert p.to_numpy(out, n).tobytes() == ref.tobytes(), rep
        # new contents at the same addresses: the replay reads them
        for f_ in frames:
            f_.mul_(-1.0)
        with st.Plan(fs, **kw) as p0:
            out0, n0, _ = p0.search(frames, ts, capacity=1 << 16)
            ref2 = p0.to_numpy(out0, n0)
        out, n, s = p.search(frames, ts, capacity=1 << 16)
        assert p.last_graph_replayed()
        assert p.to_numpy(out, n).tobytes() == ref2.tobytes()
        assert ref2.tobytes() != ref.tobytes()


def test_graph_recaptures_on_new_times_and_pointers(st):
    ds = fields(2, seed=70)
    fs = [d["field"] for d in ds]
    ts = [d["times"] for d in ds]
    raw = [d["frames"] for d in ds]
    with st.Plan(fs, use_graph=True, normalize=False) as p:
        out, n, _ = p.search([dev(r) for r in raw], ts, capacity=1 << 16)
        first = p.to_numpy(out, n)
        # shifted timestamps: new shift tables, a new capture, the oracle's result
        ts2 = [t + 0.013 * (j + 1) for j, t in enumerate(ts)]
        out, n, _ = p.search([dev(r) for r in raw], ts2, capacity=1 << 16)
        got = p.to_numpy(out, n)
        assert p.last_graph_replayed()
        for j, r in enumerate(raw):
            ref = oracle.search(r, ts2[j], fs[j], prec="fp32")
            mine = got[got["field"] == j]
            assert mine[["x", "y", "k", "n_cov"]].tolist() == \
                ref[["x", "y", "k", "n_cov"]].tolist()
        # back to the first timestamps with fresh tensors (new pointers)
        out, n, _ = p.search([dev(r) for r in raw], ts, capacity=1 << 16)
        assert p.to_numpy(out, n).tobytes() == first.tobytes()
