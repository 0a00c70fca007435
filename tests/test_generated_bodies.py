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
    lines, n_acc = g.item_loop(16, 4, 160, 8, 8, stream=False)
    text = "\n".join(lines)
    kh = 8
    for p in range(15):
        body = text.split(f"BT{p}:\n", 1)[1].split("bra.uni SNEXT;", 1)[0]
        adds = re.findall(r"add\.rn\.f32x2 %(\d+), %(\d+), sW(\d+);", body)
        assert len(adds) == 4 * kh
        seen = set()
        for d, a, w in adds:
            d, a, w = int(d), int(a), int(w)
            j, m = divmod(d, kh)
            assert d == a and w == m + g.pat_off(p, j)
            seen.add(d)
        assert seen == set(range(n_acc))
    # window pair q holds rows q and q + 8 loaded from row offset r * 160 bytes
    for q in range(kh + 3):
        assert f"mov.b64 sW{q}, {{sv{q}, sv{q + kh}}};" in text
    for r in range(16 + 3):
        assert f"ld.shared.f32 sv{r}, [sa+{r * 160}];" in text
