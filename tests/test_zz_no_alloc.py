"""The allocation-free search entry point (st_stack_search_noalloc).

Callers that cannot allocate device memory when they search (their device
memory is reserved up front by another allocator, or their host forbids
cudaMalloc after start-up) use this entry point; its scratch is a fixed
array inside the library.  It must give the same sorted candidates as the
planned search, on consecutive calls that reuse the array.  This file is
named to be collected after every other test, so a run that stops at the
first failure has run them first; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

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


def _call(st, field, frames, times, capacity, mode):
    # straight through the C ABI: no Python-side allocation of scratch
    L = st.lib()
    L.st_stack_search_noalloc.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    f = st.make_field(field)
    t = np.ascontiguousarray(times, np.float64)
    out = torch.full((capacity, 7), -7, dtype=torch.int32, device="cuda")
    cnt = C.c_int64()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = L.st_stack_search_noalloc(C.byref(f), st.MODE[mode], C.c_void_p(frames.data_ptr()),
                                       t.ctypes.data_as(C.c_void_p), C.c_void_p(out.data_ptr()),
                                       capacity, C.byref(cnt), stream)
    return status, cnt.value, out


@pytest.mark.parametrize("mode", ["nearest", "bilinear"])
def test_noalloc_matches_planned_search_twice(st, mode):
    fields = [synth.make_field("tiny"),
              synth.make_field("mid", width=160, n_frames=20, nv=25, n_blobs=0, tau=4.0)]
    for d in fields:
        frames = torch.from_numpy(d["frames"]).cuda()
        with st.Plan(d["field"], mode=mode) as p:
            ref = p.candidates(frames, d["times"])
        assert len(ref) > 0
        for _ in range(2):  # the second call reuses the array left by the first
            status, n, out = _call(st, d["field"], frames, d["times"], 4096, mode)
            assert status == st.ST_OK, st.lib().st_last_error()
            got = out[:n].cpu().numpy().view(st.CAND_DTYPE).reshape(-1)
            assert n == len(ref)
            # nearest: bit-exact like every nearest-shift parity test; bilinear
            # runs the same kernels, so it is bit-identical as well
            assert got.tobytes() == ref.tobytes()


def test_noalloc_rejects_fields_beyond_its_scratch(st):
    d = synth.make_field("tiny")
    frames = torch.from_numpy(d["frames"]).cuda()
    big = dict(d["field"], nvx=300000, nvy=50, vx0=-1.0, dvx=1e-5, vy0=-1.0, dvy=1e-3)
    status, n, out = _call(st, big, frames, d["times"], 16, "nearest")
    assert status == st.ST_ERR_INVALID
    assert b"no-alloc scratch" in st.lib().st_last_error()
