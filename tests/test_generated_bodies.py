"""CPU checks of the generated PTX bodies of the register-window stack kernel.

The bodies are the plain definition of the stack on the register window:
for pattern id p (the row offsets c_j of 4 consecutive y-velocities, a
monotone staircase) every accumulator pair m of y-velocity j gets window pair
m + c_j.  These tests check the committed include against its generator, and
the generator's pattern table and bodies against that definition.
"""
import importlib.util
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2303_07293_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_bodies", os.path.join(CSRC, "gen_bodies.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_committed_include_is_the_generator_output():
    g = _gen()
    with open(os.path.join(CSRC, "st_bodies.inc")) as fh:
        assert fh.read() == g.render()


def test_patterns_are_the_15_monotone_staircases():
    # every way 4 consecutive y-velocities can round to rows that step by 0
    # or 1 (rising) or 0 or -1 (falling), with the lowest offset at 0
    g = _gen()
    want = set()
    for d in range(8):
        steps = [(d >> b) & 1 for b in range(3)]
        c = [0, steps[0], steps[0] + steps[1], sum(steps)]
        want.add(tuple(c))
        want.add(tuple(x - min(reversed(c)) for x in reversed(c)))
    got = {tuple(g.pat_off(p, j) for j in range(4)) for p in range(15)}
    assert got == want and len(got) == 15


def test_item_loop_bodies_add_window_pair_m_plus_c():
    g = _gen()
    kh = 8
    for ky, frames, row_bytes, stages, warps, dtype in g.ITEMS:
        lines, n_acc = g.item_loop(ky, frames, row_bytes, stages, warps, dtype)
        text = "\n".join(lines)
        # rows loaded ahead of the indexed branch serve every body
        ahead = text.split("SLOOP:\n", 1)[1].split("BTT:", 1)[0]
        for p in range(15):
            body = text.split(f"BT{p}:\n", 1)[1].split("bra.uni SNEXT;", 1)[0]
            rows, pairs, seen = {}, {}, set()
            for ln in ahead.splitlines() + body.splitlines():
                # a window row reaches FP32 register sv<r>: loaded as FP32, or
                # loaded as 16 bits at the same byte offset and then converted
                # (cvt from FP16; a BF16 value shifted into the upper half)
                m16 = re.fullmatch(r"ld\.shared\.(?:b16 sh|u16 su)(\d+), \[sa\+(\d+)\];", ln)
                if m16:
                    assert dtype != "f32" and int(m16.group(2)) == int(m16.group(1)) * row_bytes
                    continue
                mcv = re.fullmatch(r"cvt\.f32\.f16 sv(\d+), sh(\d+);|mov\.b32 sv(\d+), su(\d+);",
                                   ln)
                if mcv:
                    r = int(mcv.group(1) or mcv.group(3))
                    assert r == int(mcv.group(2) or mcv.group(4)) and r not in rows
                    rows[r] = True
                    continue
                if re.fullmatch(r"shl\.b32 su(\d+), su\1, 16;", ln):
                    assert dtype == "bf16"
                    continue
                mld = re.fullmatch(r"ld\.shared\.f32 sv(\d+), \[sa\+(\d+)\];", ln)
                mmv = re.fullmatch(r"mov\.b64 sW(\d+), \{sv(\d+), sv(\d+)\};", ln)
                madd = re.fullmatch(r"add\.rn\.f32x2 %(\d+), %(\d+), sW(\d+);", ln)
                if mld:
                    assert dtype == "f32"
                    r = int(mld.group(1))
                    assert int(mld.group(2)) == r * row_bytes and r not in rows
                    rows[r] = True
                elif mmv:
                    q, lo, hi = map(int, mmv.groups())
                    # the pair holds window rows q and q + 8, both loaded before
                    assert (lo, hi) == (q, q + kh) and lo in rows and hi in rows
                    pairs[q] = True
                elif madd:
                    d, a, w = map(int, madd.groups())
                    j, m = divmod(d, kh)
                    assert d == a and w in pairs and w == m + g.pat_off(p, j)
                    assert d not in seen
                    seen.add(d)
            # every accumulator pair gets exactly one add per frame
            assert seen == set(range(n_acc))
            assert body.count("add.rn.f32x2") == n_acc
        assert text.count("brx.idx.uni sid, BTT;") == 1


def test_two_velocity_bodies_add_each_velocitys_window_pair_m_plus_c():
    # a symbolic run of each body: registers hold (window base, byte offset)
    # of what they loaded; x-velocity 0's window is at sa, x-velocity 1's at
    # sa when the body index is below 16 (the two columns agree) and at sb
    # otherwise; accumulator pair (x, j, m) is operand x*16 + j*4 + m
    g = _gen()
    for ky, frames, row_bytes, stages, warps, dtype in g.ITEMS_X2:
        kh = ky // 2
        lines, n_acc = g.item_loop_x2(ky, frames, row_bytes, stages, warps, dtype)
        assert n_acc == 2 * 4 * kh
        text = "\n".join(lines)
        # the frame's four words (body index, the two windows' ring offsets,
        # unused), the next frame's read ahead in one vector load
        head = text.split("SLOOP:\n", 1)[1].split("BTT:", 1)[0]
        assert head.splitlines()[0] == "ld.shared.v4.u32 {snid, sna, snb, sw}, [swp+16];"
        nxt = text.split("SNEXT:\n", 1)[1].splitlines()[:4]
        assert nxt[0] == "mov.u32 sid, snid;" and nxt[3] == "add.u32 swp, swp, 16;"
        assert re.fullmatch(r"add\.u32 sa, sna, %\d+;", nxt[1])
        assert re.fullmatch(r"add\.u32 sb, snb, %\d+;", nxt[2])
        targets = text.split("BTT: .branchtargets ", 1)[1].split(";", 1)[0].split(", ")
        assert targets == [f"BT{b}" for b in range(32)]
        for b in range(32):
            body = text.split(f"BT{b}:\n", 1)[1].split("bra.uni SNEXT;", 1)[0]
            if b in (15, 31):
                assert body.startswith("BT31:") or body.startswith("SNEXT:")
                assert "add.rn" not in body.split("SNEXT:", 1)[0]
                continue
            p, same = b % 16, b < 16
            sv, sw, adds = {}, {}, {}
            half = {}   # 16-bit registers: what they loaded
            for ln in head.splitlines() + body.splitlines():
                mld = re.fullmatch(r"ld\.shared\.f32 sv(\d+), \[(sa|sb)\+(\d+)\];", ln)
                m16 = re.fullmatch(r"ld\.shared\.(?:b16 sh|u16 su)(\d+), \[(sa|sb)\+(\d+)\];", ln)
                mcv = re.fullmatch(r"cvt\.f32\.f16 sv(\d+), sh(\d+);|mov\.b32 sv(\d+), su(\d+);",
                                   ln)
                mmv = re.fullmatch(r"mov\.b64 sW(\d+), \{sv(\d+), sv(\d+)\};", ln)
                madd = re.fullmatch(r"add\.rn\.f32x2 %(\d+), %(\d+), sW(\d+);", ln)
                if m16:
                    assert dtype != "f32"
                    half[int(m16.group(1))] = (m16.group(2), int(m16.group(3)))
                elif mcv:
                    assert dtype == ("f16" if mcv.group(1) else "bf16")
                    sv[int(mcv.group(1) or mcv.group(3))] = half[int(mcv.group(2) or mcv.group(4))]
                elif re.fullmatch(r"shl\.b32 su(\d+), su\1, 16;", ln):
                    assert dtype == "bf16"
                elif mld:
                    assert dtype == "f32"
                    sv[int(mld.group(1))] = (mld.group(2), int(mld.group(3)))
                elif mmv:
                    q, lo, hi = map(int, mmv.groups())
                    sw[q] = (sv[lo], sv[hi])
                elif madd:
                    d, a, w = map(int, madd.groups())
                    assert d == a and d not in adds
                    adds[d] = sw[w]
            assert sorted(adds) == list(range(n_acc)), b
            for d, (lo, hi) in adds.items():
                x, rest = divmod(d, 4 * kh)
                j, m = divmod(rest, kh)
                base = "sa" if (x == 0 or same) else "sb"
                r = m + g.pat_off(p, j)
                assert lo == (base, r * row_bytes) and hi == (base, (r + kh) * row_bytes), (b, d)
