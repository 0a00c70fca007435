"""Writes st_bodies.inc: the per-frame add bodies of the register-window
stack kernel as inline PTX, one straight-line body per staircase pattern,
entered through one indexed branch (brx.idx) on the frame's pattern id.

For tile height KY a thread holds, per y-velocity j (4 per block) and row
pair m (rows m and m + KY/2), a paired FP32 accumulator; the frame's window
is held as pairs W[q] = (window row q, window row q + KY/2).  Pattern id
gives the row offsets c_j of the 4 y-velocities (a monotone staircase, ids
0..14; id 15 is a padding frame with no adds), and its body is

    acc[j][m] = acc[j][m] + W[m + c_j]   (add.rn.f32x2)

for every j and m: the same FP32 additions, in the same frame order, as the
plain definition of the stack (one add per pixel, frame and velocity).

Run `python gen_bodies.py` after changing the patterns or tile heights; a
CPU test checks that the committed file is this script's output.
"""
import os

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "st_bodies.inc")
N_PATTERNS = 15  # ids 0..14; id 15: no-op
KYS = (16,)


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


def body(ky):
    kh = ky // 2
    n_acc = 4 * kh
    n_w = kh + 3
    wi = lambda q: n_acc + q       # operand number of W[q]
    idn = n_acc + n_w              # operand number of the pattern id
    lines = ["{", "BTT: .branchtargets " + ", ".join(f"BT{p}" for p in range(16)) + ";",
             f"brx.idx.uni %{idn}, BTT;"]
    for p in range(N_PATTERNS):
        lines.append(f"BT{p}:")
        for j in range(4):
            c = pat_off(p, j)
            for m in range(kh):
                a = j * kh + m
                lines.append(f"add.rn.f32x2 %{a}, %{a}, %{wi(m + c)};")
        lines.append("bra.uni BTE;")
    lines += ["BT15:", "BTE:", "}"]
    return lines, n_acc, n_w


def stage_loop(ky, frames, row_bytes, stream=False):
    """The frames of one ring stage for one warp, as a PTX loop: per frame,
    the warp's word (window byte offset in the ring | pattern id << 24) is
    read from shared memory, the window's ky + 3 rows are loaded into the
    pair registers W[q] = (row q, row q + ky/2), and the pattern's body is
    entered by brx.idx.  Operands: %0..%(4*ky/2 - 1) the accumulators
    (64-bit pairs, read-write), then the address of the warp's `frames`
    words and the lane's base address in the ring."""
    kh = ky // 2
    n_acc = 4 * kh
    n_w = kh + 3
    wb, lb = n_acc, n_acc + 1
    L = ["{",
         ".reg .u32 sfi, sw, sa, sid, swp;",
         f".reg .f32 sv<{ky + 3}>;",
         f".reg .b64 sW<{n_w}>;",
         ".reg .pred sp;",
         "mov.u32 sfi, 0;",
         f"mov.u32 swp, %{wb};",
         "SLOOP:",
         "ld.shared.u32 sw, [swp];",
         "and.b32 sa, sw, 16777215;",
         f"add.u32 sa, sa, %{lb};",
         "shr.u32 sid, sw, 24;"]
    if not stream:
        for r in range(ky + 3):
            L.append(f"ld.shared.f32 sv{r}, [sa+{r * row_bytes}];")
        for q in range(n_w):
            L.append(f"mov.b64 sW{q}, {{sv{q}, sv{q + kh}}};")
    L.append("BTT: .branchtargets " + ", ".join(f"BT{p}" for p in range(16)) + ";")
    L.append("brx.idx.uni sid, BTT;")
    for p in range(N_PATTERNS):
        L.append(f"BT{p}:")
        if stream and single_use:
            used = {q for q in range(n_w) for j in range(4) if 0 <= q - pat_off(p, j) < kh}
            for q in range(n_w):
                if q not in used:
                    continue
                L.append(f"ld.shared.f32 sl{q}, [sa+{q * row_bytes}];")
                L.append(f"ld.shared.f32 sh{q}, [sa+{(q + kh) * row_bytes}];")
                L.append(f"mov.b64 sW{q}, {{sl{q}, sh{q}}};")
                for j in range(4):
                    m = q - pat_off(p, j)
                    if 0 <= m < kh:
                        a = j * kh + m
                        L.append(f"add.rn.f32x2 %{a}, %{a}, sW{q};")
        elif stream:
            loaded = set()
            for q in range(n_w):
                for r in (q, q + kh):
                    if r not in loaded:
                        L.append(f"ld.shared.f32 sv{r}, [sa+{r * row_bytes}];")
                        loaded.add(r)
                L.append(f"mov.b64 sW{q}, {{sv{q}, sv{q + kh}}};")
                for j in range(4):
                    m = q - pat_off(p, j)
                    if 0 <= m < kh:
                        a = j * kh + m
                        L.append(f"add.rn.f32x2 %{a}, %{a}, sW{q};")
        else:
            for j in range(4):
                c = pat_off(p, j)
                for m in range(kh):
                    a = j * kh + m
                    L.append(f"add.rn.f32x2 %{a}, %{a}, sW{m + c};")
        L.append("bra.uni SNEXT;")
    L += ["BT15:", "SNEXT:", "add.u32 swp, swp, 4;", "add.u32 sfi, sfi, 1;",
          f"setp.lt.u32 sp, sfi, {frames};", "@sp bra.uni SLOOP;", "}"]
    return L, n_acc


STAGES = ((16, 4, 160), (12, 4, 160))  # (rows per thread, frames per stage, box row bytes)


def stage_loop_stream(ky, frames, row_bytes):
    """As stage_loop, but each pattern's body loads the window as it adds:
    at step q it loads window rows q and q + ky/2 (once each), forms the
    pair W[q] and adds it to every accumulator pair m = q - c_j, so loads
    and adds interleave and the window never sits in registers whole.  The
    next frame's word is read at the start of the body."""
    kh = ky // 2
    n_acc = 4 * kh
    n_w = kh + 3
    wb, lb = n_acc, n_acc + 1
    L = ["{",
         ".reg .u32 sfi, sw, snw, sa, sid, swp;",
         f".reg .f32 sv<{ky + 3}>;",
         f".reg .b64 sW<{n_w}>;",
         ".reg .pred sp;",
         "mov.u32 sfi, 0;",
         f"mov.u32 swp, %{wb};",
         "ld.shared.u32 sw, [swp];",
         "SLOOP:",
         "and.b32 sa, sw, 16777215;",
         f"add.u32 sa, sa, %{lb};",
         "shr.u32 sid, sw, 24;",
         "BTT: .branchtargets " + ", ".join(f"BT{p}" for p in range(16)) + ";",
         "brx.idx.uni sid, BTT;"]
    for p in range(N_PATTERNS + 1):
        L.append(f"BT{p}:")
        L.append("ld.shared.u32 snw, [swp+4];")
        if p == N_PATTERNS:
            L.append("bra.uni SNEXT;")
            continue
        loaded = set()
        for q in range(n_w):
            for r in (q, q + kh):
                if r not in loaded:
                    L.append(f"ld.shared.f32 sv{r}, [sa+{r * row_bytes}];")
                    loaded.add(r)
            L.append(f"mov.b64 sW{q}, {{sv{q}, sv{q + kh}}};")
            for j in range(4):
                m = q - pat_off(p, j)
                if 0 <= m < kh:
                    a = j * kh + m
                    L.append(f"add.rn.f32x2 %{a}, %{a}, sW{q};")
        L.append("bra.uni SNEXT;")
    L += ["SNEXT:", "mov.u32 sw, snw;", "add.u32 swp, swp, 4;", "add.u32 sfi, sfi, 1;",
          f"setp.lt.u32 sp, sfi, {frames};", "@sp bra.uni SLOOP;", "}"]
    return L, n_acc


def stage_loop_regs(ky, frames, row_bytes):
    """As stage_loop, but the warp's `frames` words of the stage come in
    registers (operands after the accumulators, then the lane's base
    address) and rotate frame by frame, so no frame waits on a word load:
    the next frame's window address and pattern id are formed before the
    current frame's body."""
    kh = ky // 2
    n_acc = 4 * kh
    n_w = kh + 3
    words = [n_acc + f for f in range(frames)]
    lb = n_acc + frames
    L = ["{",
         ".reg .u32 sfi, sa, sid, sna, snid;",
         ".reg .u32 " + ", ".join(f"sq{f}" for f in range(frames)) + ";",
         f".reg .f32 sv<{ky + 3}>;",
         f".reg .b64 sW<{n_w}>;",
         ".reg .pred sp;",
         "mov.u32 sfi, 0;"]
    for f in range(frames):
        L.append(f"mov.u32 sq{f}, %{words[f]};")
    L += ["and.b32 sa, sq0, 16777215;", f"add.u32 sa, sa, %{lb};", "shr.u32 sid, sq0, 24;",
          "SLOOP:"]
    for r in range(ky + 3):
        L.append(f"ld.shared.f32 sv{r}, [sa+{r * row_bytes}];")
    for q in range(n_w):
        L.append(f"mov.b64 sW{q}, {{sv{q}, sv{q + kh}}};")
    # the next frame's address and id (from the next word) before the body
    L += ["and.b32 sna, sq1, 16777215;", f"add.u32 sna, sna, %{lb};", "shr.u32 snid, sq1, 24;"]
    L.append("BTT: .branchtargets " + ", ".join(f"BT{p}" for p in range(16)) + ";")
    L.append("brx.idx.uni sid, BTT;")
    for p in range(N_PATTERNS):
        L.append(f"BT{p}:")
        for j in range(4):
            c = pat_off(p, j)
            for m in range(kh):
                a = j * kh + m
                L.append(f"add.rn.f32x2 %{a}, %{a}, sW{m + c};")
        L.append("bra.uni SNEXT;")
    L += ["BT15:", "SNEXT:", "mov.u32 sa, sna;", "mov.u32 sid, snid;"]
    for f in range(frames - 1):
        L.append(f"mov.u32 sq{f + 1 - 1}, sq{f + 1};" if f + 1 < frames else "")
    L += ["add.u32 sfi, sfi, 1;", f"setp.lt.u32 sp, sfi, {frames};", "@sp bra.uni SLOOP;", "}"]
    return [x for x in L if x], n_acc


def item_loop(ky, frames, row_bytes, stages, warps, wait_ns=2000000000, stream=True,
              single_use=False):
    """Every stage of one item for one warp, as one PTX block: per stage,
    wait on the stage's full barrier (all lanes, bounded by wait_ns of the
    global timer), run its frames (as stage_loop: the warp's word per frame,
    window pairs, brx.idx into the pattern bodies), then lane 0 releases the
    slot on its empty barrier.  Operands: %0.. the accumulator pairs; then
    the ring slot and phase (read-write), an error flag (out: 1 = a wait ran
    out); then the number of stages, whether the first stage's wait is
    already done, the address of this warp's words in slot 0, the lane's
    base address in the ring, and the addresses of full and empty barrier 0.
    Slot s's words are at words0 + s*warps*frames*4; barriers 8 bytes apart.
    With stream, each pattern body loads the window rows as it adds them
    (see stage_loop_stream), which keeps few window registers live; with
    single_use, a row that sits in two pairs (rows ky/2 .. ky/2 + 2) is
    loaded once for each, so every loaded register is one half of one pair
    and no register copies are needed to form the pairs."""
    kh = ky // 2
    n_acc = 4 * kh
    n_w = kh + 3
    slot, ph, err = n_acc, n_acc + 1, n_acc + 2
    nst, skip, wb0, lb, fb0, eb0 = (n_acc + 3 + i for i in range(6))
    wstride = warps * frames * 4
    L = ["{",
         ".reg .u32 sfi, sw, sa, sid, swp, sst, sbar, st0, st1;",
         f".reg .f32 sv<{ky + 3}>;"]
    if single_use:
        L.append(f".reg .f32 sl<{n_w}>, sh<{n_w}>;")
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
         f"setp.eq.u32 sp, sst, 0;",
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
         "SLOOP:",
         "ld.shared.u32 sw, [swp];",
         "and.b32 sa, sw, 16777215;",
         f"add.u32 sa, sa, %{lb};",
         "shr.u32 sid, sw, 24;"]
    if not stream:
        for r in range(ky + 3):
            L.append(f"ld.shared.f32 sv{r}, [sa+{r * row_bytes}];")
        for q in range(n_w):
            L.append(f"mov.b64 sW{q}, {{sv{q}, sv{q + kh}}};")
    L.append("BTT: .branchtargets " + ", ".join(f"BT{p}" for p in range(16)) + ";")
    L.append("brx.idx.uni sid, BTT;")
    for p in range(N_PATTERNS):
        L.append(f"BT{p}:")
        if stream and single_use:
            used = {q for q in range(n_w) for j in range(4) if 0 <= q - pat_off(p, j) < kh}
            for q in range(n_w):
                if q not in used:
                    continue
                L.append(f"ld.shared.f32 sl{q}, [sa+{q * row_bytes}];")
                L.append(f"ld.shared.f32 sh{q}, [sa+{(q + kh) * row_bytes}];")
                L.append(f"mov.b64 sW{q}, {{sl{q}, sh{q}}};")
                for j in range(4):
                    m = q - pat_off(p, j)
                    if 0 <= m < kh:
                        a = j * kh + m
                        L.append(f"add.rn.f32x2 %{a}, %{a}, sW{q};")
        elif stream:
            loaded = set()
            for q in range(n_w):
                for r in (q, q + kh):
                    if r not in loaded:
                        L.append(f"ld.shared.f32 sv{r}, [sa+{r * row_bytes}];")
                        loaded.add(r)
                L.append(f"mov.b64 sW{q}, {{sv{q}, sv{q + kh}}};")
                for j in range(4):
                    m = q - pat_off(p, j)
                    if 0 <= m < kh:
                        a = j * kh + m
                        L.append(f"add.rn.f32x2 %{a}, %{a}, sW{q};")
        else:
            for j in range(4):
                c = pat_off(p, j)
                for m in range(kh):
                    a = j * kh + m
                    L.append(f"add.rn.f32x2 %{a}, %{a}, sW{m + c};")
        L.append("bra.uni SNEXT;")
    L += ["BT15:", "SNEXT:", "add.u32 swp, swp, 4;", "add.u32 sfi, sfi, 1;",
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


ITEMS = ((16, 16, 160, 2, 16), (16, 16, 160, 2, 8), (16, 12, 160, 3, 8),
         (16, 8, 160, 4, 8), (16, 8, 160, 4, 16))  # (KY, F, row bytes, S, consumer warps)
ITEMS_WINDOW = ()
# single-use loads (no register copies for the pairs; measured no faster)
ITEMS_SINGLE = ()


def render():
    out = ["// Generated by gen_bodies.py: per-frame add bodies of the register-window",
           "// stack kernel (one per staircase pattern, entered by brx.idx).  Do not edit.",
           "#pragma once", ""]
    for ky in KYS:
        lines, n_acc, n_w = body(ky)
        out.append(f"#define ST_BODY_KY{ky} \\")
        for ln in lines:
            out.append(f'  "{ln}\\n\\t" \\')
        out.append("")
        ops = ", ".join(f'"+l"(acc[{a}])' for a in range(n_acc))
        ins = ", ".join(f'"l"(pw[{q}])' for q in range(n_w))
        out.append(f"#define ST_BODY_OPERANDS_KY{ky}(acc, pw, id) \\")
        out.append(f"  : {ops} \\")
        out.append(f'  : {ins}, "r"(id)')
        out.append("")
    for ky, frames, row_bytes in STAGES:
        lines, n_acc = stage_loop(ky, frames, row_bytes)
        out.append(f"#define ST_STAGE_KY{ky}_F{frames}_R{row_bytes} \\")
        for ln in lines:
            out.append(f'  "{ln}\\n\\t" \\')
        out.append("")
        ops = ", ".join(f'"+l"(acc[{a}])' for a in range(n_acc))
        out.append(f"#define ST_STAGE_OPERANDS_KY{ky}(acc, wb, lb) \\")
        out.append(f"  : {ops} \\")
        out.append('  : "r"(wb), "r"(lb) : "memory"')
        out.append("")
        lines, n_acc = stage_loop_stream(ky, frames, row_bytes)
        out.append(f"#define ST_STAGES_KY{ky}_F{frames}_R{row_bytes} \\")
        for ln in lines:
            out.append(f'  "{ln}\\n\\t" \\')
        out.append("")
        lines, n_acc = stage_loop_regs(ky, frames, row_bytes)
        out.append(f"#define ST_STAGEQ_KY{ky}_F{frames}_R{row_bytes} \\")
        for ln in lines:
            out.append(f'  "{ln}\\n\\t" \\')
        out.append("")
        ws = ", ".join(f'"r"(q{f})' for f in range(frames))
        out.append(f"#define ST_STAGEQ_OPERANDS_KY{ky}_F{frames}(acc, {', '.join(f'q{f}' for f in range(frames))}, lb) \\")
        out.append(f"  : {ops} \\")
        out.append(f'  : {ws}, "r"(lb) : "memory"')
        out.append("")
    for ky, frames, row_bytes, stages, warps in ITEMS:
        lines, n_acc = item_loop(ky, frames, row_bytes, stages, warps)
        out.append(f"#define ST_ITEM_KY{ky}_F{frames}_R{row_bytes}_S{stages}_W{warps} \\")
        for ln in lines:
            out.append(f'  "{ln}\\n\\t" \\')
        out.append("")
    for ky, frames, row_bytes, stages, warps in ITEMS_SINGLE:
        lines, n_acc = item_loop(ky, frames, row_bytes, stages, warps, single_use=True)
        out.append(f"#define ST_ITEMU_KY{ky}_F{frames}_R{row_bytes}_S{stages}_W{warps} \\")
        for ln in lines:
            out.append(f'  "{ln}\\n\\t" \\')
        out.append("")
    for ky, frames, row_bytes, stages, warps in ITEMS_WINDOW:
        lines, n_acc = item_loop(ky, frames, row_bytes, stages, warps, stream=False)
        out.append(f"#define ST_ITEMW_KY{ky}_F{frames}_R{row_bytes}_S{stages}_W{warps} \\")
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
