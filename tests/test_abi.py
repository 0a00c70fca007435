"""The C-ABI library loads and exports every entry point include/st.h
declares; host-side argument validation (CPU only: no compute call needs a
GPU here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(st_[a-z0-9_]+)\s*\(",
                            src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["st_plan", "st_stack_search", "st_refine", "st_free", "st_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_07293_gb300 as st
    L = st.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert st.version() == 1


def test_invalid_arguments_are_rejected_without_gpu_work():
    import paper_2303_07293_gb300 as st
    L = st.lib()
    h = C.c_void_p()
    opts = st.Opts(0, 0, 0, 0.0, 0, 0, None, 0)
    bad = st.Field(0, 10, 4, 0.0, 0.0, 1.0, 1, 0.0, 1.0, 1, 5.0, 0)
    assert L.st_plan(C.byref(bad), 1, C.byref(opts), None, C.byref(h)) == st.ST_ERR_INVALID
    assert b"width" in L.st_last_error()
    assert h.value is None
    bad2 = st.Field(8, 8, 4, 0.0, 0.0, 1.0, 1, 0.0, 1.0, 1, 5.0, 9)
    assert L.st_plan(C.byref(bad2), 1, C.byref(opts), None, C.byref(h)) == st.ST_ERR_INVALID
    assert b"min_coverage" in L.st_last_error()
    for n_frames in (0, 65536):   # frames index grid rows: at most 65535
        bad3 = st.Field(8, 8, n_frames, 0.0, 0.0, 1.0, 1, 0.0, 1.0, 1, 5.0, 0)
        assert L.st_plan(C.byref(bad3), 1, C.byref(opts), None, C.byref(h)) == st.ST_ERR_INVALID
        assert b"n_frames" in L.st_last_error()
    big = st.Field(8, 8, 4, 0.0, 0.0, 1.0, 8193, 0.0, 1.0, 8193, 5.0, 0)  # 8193^2 > 2^26
    assert L.st_plan(C.byref(big), 1, C.byref(opts), None, C.byref(h)) == st.ST_ERR_INVALID
    assert b"nvx*nvy" in L.st_last_error()
    good = st.Field(8, 8, 4, 0.0, 0.0, 1.0, 1, 0.0, 1.0, 1, 5.0, 0)
    bad_opts = st.Opts(7, 0, 0, 0.0, 0, 0, None, 0)
    assert L.st_plan(C.byref(good), 1, C.byref(bad_opts), None, C.byref(h)) == st.ST_ERR_INVALID
    assert L.st_plan(C.byref(good), 0, C.byref(opts), None, C.byref(h)) == st.ST_ERR_INVALID
    assert L.st_stack_search(None, None, None, None, 0, None) == st.ST_ERR_INVALID
    L.st_free(None)  # NULL-safe


def test_new_entry_points_validate_arguments_without_gpu_work():
    import paper_2303_07293_gb300 as st
    L = st.lib()
    P = C.c_void_p
    L.st_median_subtract.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, P, P, P]
    L.st_sum_frames.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, P, P, P]
    L.st_bin2x2.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, P, P]
    L.st_link_tracks.argtypes = [P, P, C.c_int64, C.c_int32, C.c_int32, P, C.c_int64, P]
    L.st_probe_wait_timeout.argtypes = [C.c_int32, P, P]
    fake = P(0x1000)
    assert L.st_median_subtract(None, 4, 4, 4, fake, None, None) == st.ST_ERR_INVALID
    assert L.st_median_subtract(fake, 0, 4, 4, fake, None, None) == st.ST_ERR_INVALID
    assert L.st_median_subtract(fake, 769, 4, 4, fake, None, None) == st.ST_ERR_UNSUPPORTED
    assert L.st_sum_frames(fake, 8, 4, 4, 0, None, P(0x90000), None, None) == st.ST_ERR_INVALID
    # output inside the input cube
    assert L.st_sum_frames(fake, 8, 4, 4, 2, None, P(0x1010), None, None) == st.ST_ERR_INVALID
    assert L.st_bin2x2(fake, 2, 8, 8, P(0x1020), None) == st.ST_ERR_INVALID
    cnt = C.c_int64()
    assert L.st_link_tracks(None, fake, 1, 2, 1, fake, 1, C.byref(cnt)) == st.ST_ERR_INVALID
    f = C.c_int32()
    d = C.c_double()
    assert L.st_probe_wait_timeout(0, C.byref(f), C.byref(d)) == st.ST_ERR_INVALID
    assert L.st_probe_wait_timeout(3000000, C.byref(f), C.byref(d)) == st.ST_ERR_INVALID


def test_binding_rejects_host_tensors_before_the_library():
    # the binding's marshalling checks run before any library call: CPU
    # tensors (or wrong dtypes / layouts) never reach the C ABI
    import torch
    import paper_2303_07293_gb300 as st
    cpu = torch.zeros((4, 8, 8), dtype=torch.float32)
    with pytest.raises(ValueError):
        st.median_subtract(cpu)
    with pytest.raises(ValueError):
        st.sum_frames(cpu, np.arange(4.0), 2)
    with pytest.raises(ValueError):
        st.bin2x2(cpu)
    with pytest.raises(ValueError):
        st.search_noalloc(dict(width=8, height=8, n_frames=4, t_ref=0.0, vx0=0.0, dvx=1.0,
                               nvx=1, vy0=0.0, dvy=1.0, nvy=1, snr_threshold=5.0),
                          cpu, np.arange(4.0))


def test_header_is_c99_and_its_layouts_match_the_binding(tmp_path):
    # the header compiles as strict C99, and every struct the binding mirrors
    # (ctypes structures, numpy record dtypes) has the same size and field
    # offsets as the C compiler gives it
    import shutil
    import subprocess
    import paper_2303_07293_gb300 as st
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    layouts = {
        "st_field": ([f for f, _ in st.Field._fields_], C.sizeof(st.Field),
                     [getattr(st.Field, f).offset for f, _ in st.Field._fields_]),
        "st_opts": ([f for f, _ in st.Opts._fields_], C.sizeof(st.Opts),
                    [getattr(st.Opts, f).offset for f, _ in st.Opts._fields_]),
        "st_candidate": (list(st.CAND_DTYPE.names), st.CAND_DTYPE.itemsize,
                         [st.CAND_DTYPE.fields[n][1] for n in st.CAND_DTYPE.names]),
        "st_track": (list(st.TRACK_DTYPE.names), st.TRACK_DTYPE.itemsize,
                     [st.TRACK_DTYPE.fields[n][1] for n in st.TRACK_DTYPE.names]),
        "st_refined": (list(st.REFINED_DTYPE.names),
                       st.REFINED_DTYPE.itemsize,
                       [st.REFINED_DTYPE.fields[n][1] for n in st.REFINED_DTYPE.names]),
    }
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "st.h"', "int main(void) {"]
    for t, (names, _, _) in layouts.items():
        lines.append(f'  printf("{t} %zu", sizeof({t}));')
        for n in names:
            lines.append(f'  printf(" %zu", offsetof({t}, {n}));')
        lines.append('  printf("\\n");')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I",
                    os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {ln.split()[0]: [int(v) for v in ln.split()[1:]] for ln in out if ln.strip()}
    for t, (names, size, offs) in layouts.items():
        assert got[t][0] == size, (t, got[t][0], size)
        assert got[t][1:] == offs, (t, names, got[t][1:], offs)
