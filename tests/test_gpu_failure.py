"""Failure detection on the GPU without a fault: every wait of the library's
pipelines is bounded in time and reports that it ran out instead of hanging.
A probe waits on an mbarrier phase that nothing completes; the wait must give
up near its limit, report it, and leave the context usable (a search right
after gives the oracle's result)."""
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


@pytest.mark.parametrize("limit_us", [1000, 100000])
def test_bounded_wait_gives_up_and_context_stays_usable(st, limit_us):
    timed_out, waited = st.probe_wait_timeout(limit_us)
    assert timed_out
    assert limit_us <= waited <= limit_us + 500000      # gave up after the limit, not much later
    d = synth.make_field("tiny")
    with st.Plan(d["field"]) as p:
        got = p.candidates(torch.from_numpy(d["frames"]).cuda(), d["times"])
    ref = oracle.search(d["frames"], d["times"], d["field"], prec="fp32")
    assert got[["x", "y", "k"]].tolist() == ref[["x", "y", "k"]].tolist()
