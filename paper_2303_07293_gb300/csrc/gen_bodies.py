"""Writes st_bodies.inc: the consumer loop of the register-window stack
kernel as inline PTX, one block per (rows per thread, frames per stage, ring
stages, consumer warps) the kernel instantiates.

For tile height KY a thread holds, per y-velocity j (4 per block) and row
pair m (rows m and m + KY/2), a paired FP32 accumulator; the frame's window
is held as pairs W[q] = (window row q, window row q + KY/2).  A frame's
pattern id gives the row offsets c_j of the 4 y-velocities (a monotone
staircase, ids 0..14; id 15 is a padding frame with no adds), and its body is

    acc[j][m] = acc[j][m] + W[m + c_j]   (add.rn.f32x2)

for every j and m: the same FP32 additions, in the same frame order, as the
plain definition of the stack (one add per pixel, frame and velocity).  A
body is entered by one indexed branch (brx.idx) on the id and loads the
window rows as it adds them, only those its pattern uses.

Run `python gen_bodies.py` after changing the patterns or the instantiated
shapes; a CPU test checks that the committed file is this script's output.
"""
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "st_bodies.inc")
N_PATTERNS = 15  # ids 0..14; id 15: no-op
PRE = 3          # window pairs loaded ahead of the indexed branch
PRE_X2 = 3       # the same, two x-velocities a thread
# storage types: PTX load of one window element and its conversion to FP32
# (FP16 by cvt; a BF16 value is the upper half of its FP32 value)
DTYPES = {
    "f32": ("ld.shared.f32 sv{r}, [sa+{o}];", None),
    "f16": ("ld.shared.b16 sh{r}, [sa+{o}];", "cvt.f32.f16 sv{r}, sh{r};"),
    "bf16": ("ld.shared.u16 su{r}, [sa+{o}];", "shl.b32 su{r}, su{r}, 16;\nmov.b32 sv{r}, su{r};"),
}
# (rows per thread, frames per stage, box row bytes, ring stages, consumer warps, storage):
# FP32 boxes are 40 wide (160 B rows), 16-bit boxes 48 wide (96 B rows)
ITEMS = ((16, 16, 160, 2, 16, "f32"), (16, 16, 160, 2, 8, "f32"), (16, 12, 160, 3, 8, "f32"),
         (16, 8, 160, 4, 8, "f32"), (16, 8, 160, 4, 16, "f32"),
         (16, 16, 96, 2, 16, "f16"), (16, 16, 96, 2, 8, "f16"),
         (16, 16, 96, 2, 16, "bf16"), (16, 16, 96, 2, 8, "bf16"))


def pat_off(pid, j):
    """Row offset of y-velocity j in pattern pid (minimum offset 0): ids 0..7
    rise by steps (bit 0, bit 1, bit 2); ids 8..14 fall by the steps of
    t = id - 7 read from the other end."""
    if pid < 8:
        s = [(pid >> b) & 1 for b in range(3)]
        return [0, s[0], s[0] + s[1], s[0] + s[1] + s[2]][j]
    t = pid - 7
    s = [(t >> b) & 1 for b in range(3)]
    return [s[0] + s[1] + s[2], s[1] + s[2], s[2], 0][j]


def pattern_body(p, ky, row_bytes, dtype="f32", preloaded=()):
    """PTX of pattern p's body: at step q, load window rows q and q + ky/2
    (each row once, converted to FP32 for 16-bit storage), form W[q] and add
    it to every accumulator pair m = q - c_j; steps whose pair no y-velocity
    uses are left out."""
    ld, cvt = DTYPES[dtype]
    kh = ky // 2
    used = {q for q in range(kh + 3) for j in range(4) if 0 <= q - pat_off(p, j) < kh}
    loaded = set(preloaded)
    L = []
    for q in range(kh + 3):
        if q not in used:
            continue
        for r in (q, q + kh):
            if r not in loaded:
                L.append(ld.format(r=r, o=r * row_bytes))
                if cvt:
                    L += cvt.format(r=r).split("\n")
                loaded.add(r)
        L.append(f"mov.b64 sW{q}, {{sv{q}, sv{q + kh}}};")
        for j in range(4):
            m = q - pat_off(p, j)
            if 0 <= m < kh:
                a = j * kh + m
                L.append(f"add.rn.f32x2 %{a}, %{a}, sW{q};")
    return L


def item_loop(ky, frames, row_bytes, stages, warps, dtype="f32", wait_ns=2000000000):
    """Every stage of one item for one warp, as one PTX block: per stage,
    wait on the stage's full barrier (all lanes, bounded by wait_ns of the
    global timer), run its frames (per frame: the warp's word, the byte
    offset of its window in the ring with the pattern id in the top byte,
    read one frame ahead; brx.idx into the pattern's body), then lane 0
    releases the slot on its empty barrier.  The read ahead of a stage's last
    frame touches the word after the warp's words (the next warp's, or one
    word of padding after the last).  Operands: %0.. the accumulator pairs; then the ring slot
    and phase (read-write), an error flag (out: 1 = a wait ran out); then the
    number of stages, whether the first stage's wait is already done, the
    address of this warp's words in slot 0, the lane's base address in the
    ring, and the addresses of full and empty barrier 0.  Slot s's words are
    at words0 + s*warps*frames*4; barriers 8 bytes apart."""
    kh = ky // 2
    n_acc = 4 * kh
    n_w = kh + 3
    slot, ph, err = n_acc, n_acc + 1, n_acc + 2
    nst, skip, wb0, lb, fb0, eb0 = (n_acc + 3 + i for i in range(6))
    wstride = warps * frames * 4
    L = ["{",
         ".reg .u32 sfi, sw, snw, sa, sid, swp, sst, sbar, st0, st1;",
         f".reg .f32 sv<{ky + 3}>;"]
    if dtype == "f16":
        L.append(f".reg .b16 sh<{ky + 3}>;")
    if dtype == "bf16":
        L.append(f".reg .u32 su<{ky + 3}>;")
    L += [f".reg .b64 sW<{n_w}>;",
         ".reg .pred sp, swt, sall, slane, sany;",
         f"mov.u32 %{err}, %laneid;",
         f"setp.eq.u32 slane, %{err}, 0;",
         f"mov.u32 %{err}, 0;",
         "mov.u32 sst, 0;",
         f"setp.ge.u32 sp, sst, %{nst};",
         "@sp bra.uni IEND;",
         "ISTAGE:",
         # the stage's full barrier (skipped for the first stage when asked)
         "setp.eq.u32 sp, sst, 0;",
         f"setp.ne.and.u32 sp, %{skip}, 0, sp;",
         "@sp bra.uni IRUN;",
         f"mad.lo.u32 sbar, %{slot}, 8, %{fb0};",
         f"mbarrier.try_wait.parity.shared::cta.b64 swt, [sbar], %{ph};",
         "vote.sync.all.pred sall, swt, 0xffffffff;",
         "@sall bra.uni IRUN;",
         "mov.u32 st0, %globaltimer_lo;",
         "IWAIT:",
         # suspend in the barrier (up to 20 us a try) rather than spin
         f"mbarrier.try_wait.parity.shared::cta.b64 swt, [sbar], %{ph}, 20000;",
         "vote.sync.all.pred sall, swt, 0xffffffff;",
         "@sall bra.uni IRUN;",
         "mov.u32 st1, %globaltimer_lo;",
         "sub.u32 st1, st1, st0;",  # modulo 2^32 ns: exact below 4.29 s
         f"setp.gt.u32 sp, st1, {wait_ns};",
         "vote.sync.any.pred sany, sp, 0xffffffff;",
         "@!sany bra.uni IWAIT;",
         f"mov.u32 %{err}, 1;",
         "bra.uni IEND;",
         "IRUN:",
         f"mad.lo.u32 swp, %{slot}, {wstride}, %{wb0};",
         "mov.u32 sfi, 0;",
         # the frame's word was read by the previous frame (the first here);
         # the next frame's word is read before the indexed branch
         "ld.shared.u32 sw, [swp];",
         "SLOOP:",
         "and.b32 sa, sw, 16777215;",
         f"add.u32 sa, sa, %{lb};",
         "shr.u32 sid, sw, 24;",
         "ld.shared.u32 snw, [swp+4];"]
    # rows every pattern uses (window pairs 0..PRE-1: the y-velocity with
    # offset 0 adds them), loaded before the indexed branch so their latency
    # overlaps it
    pre = [r for q in range(PRE) for r in (q, q + kh)]
    ld, cvt = DTYPES[dtype]
    for r in pre:
        L.append(ld.format(r=r, o=r * row_bytes))
        if cvt:
            L += cvt.format(r=r).split("\n")
    L += ["BTT: .branchtargets " + ", ".join(f"BT{p}" for p in range(16)) + ";",
          "brx.idx.uni sid, BTT;"]
    for p in range(N_PATTERNS):
        L.append(f"BT{p}:")
        L += pattern_body(p, ky, row_bytes, dtype, preloaded=pre)
        L.append("bra.uni SNEXT;")
    L += ["BT15:", "SNEXT:", "mov.u32 sw, snw;", "add.u32 swp, swp, 4;", "add.u32 sfi, sfi, 1;",
          f"setp.lt.u32 sp, sfi, {frames};", "@sp bra.uni SLOOP;",
          # release the slot (every lane's reads are done), next slot
          "bar.warp.sync 0xffffffff;",
          f"mad.lo.u32 sbar, %{slot}, 8, %{eb0};",
          "@slane mbarrier.arrive.shared::cta.b64 _, [sbar];",
          f"add.u32 %{slot}, %{slot}, 1;",
          f"setp.eq.u32 sp, %{slot}, {stages};",
          f"@sp mov.u32 %{slot}, 0;",
          f"@sp xor.b32 %{ph}, %{ph}, 1;",
          "add.u32 sst, sst, 1;",
          f"setp.lt.u32 sp, sst, %{nst};",
          "@sp bra.uni ISTAGE;",
          "IEND:", "}"]
    return L, n_acc


# two x-velocities a thread (rows per thread, frames per stage, box row bytes,
# ring stages, consumer warps, storage): 32 accumulator pairs, as for 16
# rows; the boxes of 16 x-velocities are 48 FP32 (192 B rows) or 56 16-bit
# values (112 B rows) wide
ITEMS_X2 = ((8, 16, 192, 2, 8, "f32"), (8, 16, 192, 2, 16, "f32"),
            (8, 16, 112, 2, 8, "f16"), (8, 16, 112, 2, 8, "bf16"))


def pattern_body_x2(p, ky, row_bytes, same, dtype="f32", preloaded=()):
    """Body of pattern p for a thread with two x-velocities (accumulator pair
    (x, j, m) is operand x*4*ky/2 + j*ky/2 + m; window pairs (q, q + ky/2)).
    same: both x-velocities read the window at sa, each pair feeding both
    velocities' accumulators; otherwise x-velocity 0 reads at sa, then
    x-velocity 1 at sb."""
    ld, cvt = DTYPES[dtype]
    kh = ky // 2
    used = {q for q in range(kh + 3) for j in range(4) if 0 <= q - pat_off(p, j) < kh}
    L = []
    for x, addr in ((0, "sa"), (1, "sb")):
        if same and x == 1:
            break
        loaded = set(preloaded) if x == 0 else set()
        for q in range(kh + 3):
            if q not in used:
                continue
            for r in (q, q + kh):
                if r not in loaded:
                    L.append(ld.format(r=r, o=r * row_bytes).replace("[sa+", f"[{addr}+"))
                    if cvt:
                        L += cvt.format(r=r).split("\n")
                    loaded.add(r)
            L.append(f"mov.b64 sW{q}, {{sv{q}, sv{q + kh}}};")
            for xx in ((0, 1) if same else (x,)):
                for j in range(4):
                    m = q - pat_off(p, j)
                    if 0 <= m < kh:
                        a = xx * 4 * kh + j * kh + m
                        L.append(f"add.rn.f32x2 %{a}, %{a}, sW{q};")
    return L


def item_loop_x2(ky, frames, row_bytes, stages, warps, dtype="f32", wait_ns=2000000000):
    """As item_loop, for a thread with two adjacent x-velocities.  A frame's
    words are four: the body index (the pattern id, plus 16 when the two
    x-velocities read different columns: 0..14 and 16..30; 15 and 31: no
    adds), the byte offsets in the ring of x-velocity 0's and x-velocity 1's
    windows, and one unused word; the next frame's four are read in one
    vector load before the indexed branch.  When the two columns agree (most
    frames: adjacent velocities round to the same shift) one window feeds
    both velocities' adds.  Slot s's words are at words0 + s*warps*frames*16."""
    kh = ky // 2
    n_acc = 2 * 4 * kh
    lb = n_acc + 3 + 3
    # the stage and barrier logic of the one-velocity loop, with its
    # operands after the accumulators moved up by the extra 4*kh pairs, its
    # words four times as wide
    single, _ = item_loop(ky, frames, row_bytes, stages, warps, dtype, wait_ns=wait_ns)
    base = 4 * kh

    def renum(ln):
        return re.sub(r"%(\d+)", lambda m_: f"%{int(m_.group(1)) + (n_acc - base)}"
                      if int(m_.group(1)) >= base else m_.group(0), ln)
    head = [renum(ln) for ln in single[:single.index("SLOOP:")]]
    tail = [renum(ln) for ln in single[single.index("SNEXT:"):]]
    head[1] = head[1].replace("sfi, sw, snw, sa, sid,", "sfi, sw, sa, sb, sid, sna, snb, snid,")
    i = head.index("ld.shared.u32 sw, [swp];")
    head[i:i + 1] = ["ld.shared.v4.u32 {sid, sa, sb, sw}, [swp];",
                     f"add.u32 sa, sa, %{lb};",
                     f"add.u32 sb, sb, %{lb};"]
    i = [k for k, ln in enumerate(head) if ln.startswith("mad.lo.u32 swp,")][0]
    head[i] = re.sub(r", (\d+), ", lambda m_: f", {int(m_.group(1)) * 4}, ", head[i])
    i = tail.index("mov.u32 sw, snw;")
    tail[i:i + 2] = ["mov.u32 sid, snid;", f"add.u32 sa, sna, %{lb};", f"add.u32 sb, snb, %{lb};",
                     "add.u32 swp, swp, 16;"]
    pre = [r for q in range(PRE_X2) for r in (q, q + kh)]
    L = head + ["SLOOP:", "ld.shared.v4.u32 {snid, sna, snb, sw}, [swp+16];"]
    ld, cvt = DTYPES[dtype]
    for r in pre:
        L.append(ld.format(r=r, o=r * row_bytes))
        if cvt:
            L += cvt.format(r=r).split("\n")
    L += ["BTT: .branchtargets " + ", ".join(f"BT{p}" for p in range(32)) + ";",
          "brx.idx.uni sid, BTT;"]
    for same in (True, False):
        for p in range(N_PATTERNS):
            L.append(f"BT{p + (0 if same else 16)}:")
            L += pattern_body_x2(p, ky, row_bytes, same, dtype, preloaded=pre)
            L.append("bra.uni SNEXT;")
    L += ["BT15:", "BT31:"] + tail
    return L, n_acc


def render():
    out = ["// Generated by gen_bodies.py: the consumer loop of the register-window",
           "// stack kernel (pattern bodies entered by brx.idx).  Do not edit.",
           "#pragma once", ""]
    for ky, frames, row_bytes, stages, warps, dtype in ITEMS:
        lines, n_acc = item_loop(ky, frames, row_bytes, stages, warps, dtype)
        sfx = "" if dtype == "f32" else "_" + dtype.upper()
        out.append(f"#define ST_ITEM_KY{ky}_F{frames}_R{row_bytes}_S{stages}_W{warps}{sfx} \\")
        for ln in lines:
            out.append(f'  "{ln}\\n\\t" \\')
        out.append("")
    for ky, frames, row_bytes, stages, warps, dtype in ITEMS_X2:
        lines, n_acc = item_loop_x2(ky, frames, row_bytes, stages, warps, dtype)
        sfx = "" if dtype == "f32" else "_" + dtype.upper()
        out.append(f"#define ST_ITEMX2_KY{ky}_F{frames}_R{row_bytes}_S{stages}_W{warps}{sfx} \\")
        for ln in lines:
            out.append(f'  "{ln}\\n\\t" \\')
        out.append("")
    for ky in sorted({k[0] for k in ITEMS}):
        n_acc = 4 * (ky // 2)
        ops = ", ".join(f'"+l"(acc[{a}])' for a in range(n_acc))
        out.append(f"#define ST_ITEM_OPERANDS_KY{ky}(acc, slot, ph, err, nst, skip, wb0, lb, fb0, eb0) \\")
        out.append(f'  : {ops}, "+r"(slot), "+r"(ph), "=r"(err) \\')
        out.append('  : "r"(nst), "r"(skip), "r"(wb0), "r"(lb), "r"(fb0), "r"(eb0) : "memory"')
        out.append("")
    return "\n".join(out)


if __name__ == "__main__":
    with open(OUT, "w") as fh:
        fh.write(render())
    print(OUT)
