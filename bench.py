"""Benchmark of the synthetic-tracking search (one JSON line on rank 0).

A step is one full search of one synthetic field through the library:
shift tables, (optional) normalisation, shift-and-stack over the whole
velocity grid, threshold, local maxima and the sorted candidate list.
Default workload: a SPECULOOS-shaped field, 256 frames of 2048 x 2048 px at
50 s cadence, velocity grid +-100 px/h step 0.25 px/h (801 x 801).

Metric: G pixel*frame*velocity adds/s = P*N*N_v / step time (N_v = 641 601),
with fields/hr beside it.  The frame cube (4 GiB in FP32) is larger than L2,
so no flush is needed between steps.

--impl reference times the CPU oracle (the only baseline: the paper's own
tracker is closed software) on a bounded slab of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

T_START = time.perf_counter()
ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "speculoos": dict(name="speculoos", desc="2048x2048x256, 801x801 velocity grid"),
    "mid": dict(name="mid", desc="1024x1024x64, 161x161 velocity grid"),
    "tiny": dict(name="tiny", desc="128x128x16, 21x21 velocity grid"),
    "batched": dict(name="batched", desc="24 fields: N in [40,400], sizes {512,1024,2048}^2, "
                    "baselines 1-8 h, grid step 1 px/baseline, +-60 px/h, one plan"),
    "refine": dict(name="refine", desc="4096 candidates of a 2048x2048x300 field's 801x801 grid "
                   "search, 64x64 cutouts, 20 Adam steps"),
    "multinight": dict(name="multinight", desc="2 nights x 64 frames of 1024x1024 (2 min cadence, "
                       "24 h apart), grid +-5 px/h at 1 px over the baseline (243x243)"),
    "front": dict(name="speculoos", desc="front end on the 2048x2048x256 field: median star "
                  "removal over groups of 50 frames overlapping by 5, sums of every 13 frames, "
                  "2x2 binning"),
}
METRIC = "G pixel*frame*velocity adds/s (2048x2048x256, 801x801 grid)"

# DRAM bytes (read + write) of one stack-kernel launch, from one ncu capture
# of `--metrics dram__bytes_read.sum,dram__bytes_write.sum` (profiles/
# stack_speculoos_2048x256_traffic.md), keyed by workload, storage, sampling
# and the kernel variant that ran, with the SHA-1 prefix of the kernel's code
# it was taken on (k_stack_fast.cu and its generated PTX bodies, comments and
# blank lines removed, so only a change of the code itself retires the
# figure): reported only while the code is that one.
STACK_TRAFFIC = {
    ("speculoos", "f32", "nearest", "float_ky8_s2_f16_cpfalse_o48_h1"):
        (45.867799296e9 + 370.29248e6, "119452094ca3"),
}


def stack_source_sha():
    import hashlib
    code = []
    for name in ("k_stack_fast.cu", "st_bodies.inc"):
        path = os.path.join(ROOT, "paper_2303_07293_gb300", "csrc", name)
        with open(path) as fh:
            for line in fh:
                line = line.split("//", 1)[0].strip()
                if line:
                    code.append(line)
    return hashlib.sha1("\n".join(code).encode()).hexdigest()[:12]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="speculoos", choices=list(WORKLOADS))
    ap.add_argument("--storage", default=None, choices=["f32", "f16", "bf16"],
                    help="frame storage (default: f16 for the batched workload, else f32)")
    ap.add_argument("--graph", type=int, default=None,
                    help="capture the search in a CUDA graph (default: 1 for batched)")
    ap.add_argument("--mode", default="nearest", choices=["nearest", "bilinear"])
    ap.add_argument("--normalize", type=int, default=1)
    ap.add_argument("--cr-clip", type=float, default=10.0,
                    help="zero |I| > cr_clip sigma after normalisation (cosmic-ray removal)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1,
                    help="searches timed end to end through the host-buffer entry point")
    ap.add_argument("--time-budget", type=float, default=1500.0,
                    help="wall-clock seconds the whole run aims to stay within: warm-up "
                         "steps beyond 3 and then timed steps are cut (and reported) when "
                         "the measured step time would overrun it")
    ap.add_argument("--width", type=int, default=None,
                    help="override the workload's frame size (square), e.g. for a profiling case")
    ap.add_argument("--frames", type=int, default=None, help="override the frame count")
    ap.add_argument("--nv", type=int, default=None, help="override the grid size per axis")
    ap.add_argument("--tracks", action="store_true",
                    help="after timing: link the candidates into tracks and time it")
    ap.add_argument("--precision", action="store_true",
                    help="after timing: stack error vs the FP64 oracle at sampled candidates "
                         "and recovery of the injected movers (single-field workloads)")
    ap.add_argument("--optimizer", default="adam", choices=["adam", "gn"],
                    help="refine workload: Adam or damped Gauss-Newton steps")
    ap.add_argument("--tile", type=int, default=-1,
                    help="-1 autotune (first warm-up step), 0 default, 1 direct-gather, 2.. variant")
    args = ap.parse_args()
    if args.storage is None:
        args.storage = "f16" if args.workload == "batched" else "f32"
    if args.graph is None:
        args.graph = 1 if args.workload == "batched" else 0
    return args


class Clocks:
    """nvidia-smi sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def oracle_baseline(d, seconds, mode="nearest"):
    """Oracle (as it stands: FP32-sequential nearest, FP64 bilinear) on a slab
    of velocity planes of the same field; returns (adds/s, cores, sample
    description, elapsed)."""
    import oracle
    oracle.lib()  # build/load outside the timed region
    f = d["field"]
    N, H, W = d["frames"].shape
    cores = oracle.num_threads()
    fr = np.nan_to_num(d["frames"], nan=0.0)
    nk = f["nvx"] * f["nvy"]
    k0 = nk // 2 - cores // 2
    prec = "fp64" if mode == "bilinear" else "fp32"
    # one untimed round of `cores` planes (thread start-up, caches), then
    # rounds of planes until the sample has taken `seconds`
    t0 = time.perf_counter()
    oracle.search(fr, d["times"], f, mode=mode, prec=prec, k_begin=k0, k_end=k0 + cores)
    # rounds of at least ~0.5 s, so per-call set-up does not count
    chunk = cores * max(1, int(0.5 / max(time.perf_counter() - t0, 1e-6)))
    k1 = k0 + cores
    el = 0.0
    while el < seconds and k1 < nk:
        k_next = min(nk, k1 + chunk)
        t0 = time.perf_counter()
        oracle.search(fr, d["times"], f, mode=mode, prec=prec, k_begin=k1, k_end=k_next)
        el += time.perf_counter() - t0
        k1 = k_next
    n_planes = k1 - (k0 + cores)
    adds = float(W * H * N) * n_planes
    kind = "FP64 bilinear" if mode == "bilinear" else "FP32-sequential nearest"
    return adds / el, cores, (f"{n_planes} velocity planes (k {k0 + cores}..{k1 - 1}) of the "
                              f"full {W}x{H}x{N} field, {kind} oracle"), el


BATCH = 24


def field_for(args, rank, world):
    """The rank's input: for the batched workload its share of the 24 fields
    (longest-work-first assignment: total work fixed, strong scaling), else a
    field of its own (weak scaling)."""
    import synth
    w = WORKLOADS[args.workload]["name"]
    base = synth.BASE_SEED + {"tiny": 1, "mid": 2, "speculoos": 3, "batched": 4, "refine": 5,
                              "multinight": 6}[w]
    if w == "batched":
        from paper_2303_07293_gb300 import shard
        specs = [synth.batched_field(base, j) for j in range(BATCH)]
        mine = shard.assign_fields(specs, world)[rank]
        total = float(sum(shard.field_work(f) for f in specs))
        return [synth.make_field(w, seed=base, index=j) for j in mine], total
    kw = {k: v for k, v in (("width", args.width), ("n_frames", args.frames), ("nv", args.nv))
          if v is not None}
    return synth.make_field(w, seed=base + 100000 * rank, **kw), None


def l2_statement(ds, storage):
    """How the timed steps stand to the 129 MB L2: the cube the stack kernel
    reads (every field of the rank, in the storage type) against it."""
    mb = sum(x["frames"].size for x in ds) * (4 if storage == "f32" else 2) / 1e6
    if mb > 129.0:
        return f"inputs larger than L2 (stored frame cube {mb:.0f} MB > 129 MB)"
    return f"inputs smaller than L2 (stored frame cube {mb:.1f} MB): steps reuse L2"


def precision_report(args, d, cand):
    """Stack error of the reported candidates against the FP64 oracle on the
    same normalised frames (so FP16/BF16 storage rounding is included), in
    sigma units of the stack (S / sqrt(n_cov)), and the fraction of injected
    movers with a candidate within 2 px and one grid step of the truth."""
    import oracle
    import synth
    f = d["field"]
    rng = np.random.default_rng(7)
    norm = oracle.normalize(d["frames"], cr_clip=args.cr_clip if args.normalize else 0.0)[0] \
        if args.normalize else np.nan_to_num(d["frames"])
    n = len(cand)
    idx = rng.choice(n, min(2000, n), replace=False) if n else np.zeros(0, int)
    xyk = np.stack([cand["x"][idx], cand["y"][idx], cand["k"][idx]], axis=1)
    S64, C64 = oracle.stack_points(norm, d["times"], f, xyk, mode=args.mode, prec="fp64")
    err = (cand["stack"][idx].astype(np.float64) - S64) / np.sqrt(np.maximum(C64, 1))
    rel = np.abs(cand["stack"][idx] - S64) / np.maximum(np.abs(S64), np.sqrt(f["n_frames"]))
    nvx = f["nvx"]
    ca, cb = cand["k"] % nvx, cand["k"] // nvx
    found = 0
    for m in d["truth"]:
        a, b, _ = synth.velocity_index(f, m[2], m[3])
        hit = (np.abs(cand["x"] - m[0]) <= 2) & (np.abs(cand["y"] - m[1]) <= 2) & \
              (np.abs(ca - a) <= 1) & (np.abs(cb - b) <= 1)
        found += bool(hit.any())
    return {"storage": args.storage, "points": int(len(idx)),
            "err_rms_sigma": float(np.sqrt(np.mean(err ** 2))) if len(idx) else None,
            "err_max_sigma": float(np.max(np.abs(err))) if len(idx) else None,
            "err_max_rel": float(np.max(rel)) if len(idx) else None,
            "movers": int(len(d["truth"])), "recovered": int(found),
            "recovery_rate": found / max(len(d["truth"]), 1)}


REFINE_N, REFINE_STEPS, REFINE_CUT = 4096, 20, 64


def refine_units(N, steps=REFINE_STEPS):
    """Bilinear cutout samples of one refinement call: candidates x cutout
    pixels x frames x (steps + 1) objective evaluations."""
    return float(REFINE_N) * REFINE_CUT * REFINE_CUT * N * (steps + 1)


def refine_reference(args, d, config):
    """The FP64 refinement oracle on a bounded sample of the candidates (one
    objective-and-gradient evaluation each, at the injected movers' grid
    points), scaled to samples/s."""
    import oracle
    oracle.lib()
    fr = np.nan_to_num(d["frames"], nan=0.0)
    N = fr.shape[0]
    tr = d["truth"]
    cores = oracle.num_threads()
    th = np.array([[m[2], m[3], m[0], m[1], m[4]] for m in tr], np.float64)
    ce = np.rint(th[:, 2:4]).astype(np.int32)
    t0 = time.perf_counter()
    oracle.refine_eval(fr, d["times"], d["field"]["t_ref"], th[:cores], ce[:cores])
    one = (time.perf_counter() - t0) / min(cores, len(th))
    n = int(max(1, min(len(th), max(1.0, args.cpu_seconds / 3) / max(one, 1e-6))))
    vals = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.refine_eval(fr, d["times"], d["field"]["t_ref"], th[:n], ce[:n])
        el = time.perf_counter() - t0
        if s >= args.warmup:
            vals.append(n * REFINE_CUT * REFINE_CUT * N / el / 1e9)
    v = float(np.median(vals))
    sample = (f"{n} candidates x one FP64 objective+gradient evaluation of a {REFINE_CUT}^2 "
              f"cutout over {N} frames")
    print(json.dumps({
        "impl": "reference", "metric": REFINE_METRIC, "value": v, "unit": "G samples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config,
        "cpu_baseline": {"value": v, "unit": "G samples/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "G samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


REFINE_METRIC = ("G bilinear cutout samples/s (4096 candidates x 64^2 px x 300 frames x 21 "
                 "evaluations)")


def bench_refine(args, d, config, dev, world, rank, local):
    """Row a9: st_refine on the 4096 highest-SNR candidates of the field's
    grid search (the search itself is set-up, not timed)."""
    import torch
    import paper_2303_07293_gb300 as st
    f = d["field"]
    N, H, W = d["frames"].shape
    stream = torch.cuda.current_stream(dev)
    frames = torch.from_numpy(d["frames"]).to(dev)
    plan = st.Plan(f, storage=args.storage, normalize=bool(args.normalize),
                   cr_clip=args.cr_clip if args.normalize else 0.0, tile=args.tile,
                   pending_capacity=1 << 24, stream=stream)
    cap = 1 << 22
    out = torch.empty((cap, 7), dtype=torch.int32, device=dev)
    _, n, status = plan.search(frames, d["times"], capacity=cap, out=out)
    if status != st.ST_OK:
        raise RuntimeError(f"search status {status}")
    recs = out[:n].cpu().numpy().view(st.CAND_DTYPE).reshape(-1)
    order = np.argsort(-recs["snr"], kind="stable")[:REFINE_N]
    top = recs[order]
    if len(top) < REFINE_N:  # a quiet field: repeat the list to the batch size
        top = np.resize(top, REFINE_N)
    cands = torch.from_numpy(np.ascontiguousarray(top).view(np.int32).reshape(-1, 7)).to(dev)

    def step():
        return plan.refine(cands, steps=REFINE_STEPS, optimizer=args.optimizer)

    for _ in range(args.warmup):
        rec = step()
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        rec = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_step = ev0.elapsed_time(ev1) / 1e3 / args.steps
    if world > 1:
        tt = torch.tensor([t_step], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_step = float(tt.item())
    units = refine_units(N)
    value = units * world / t_step / 1e9
    # end to end: candidates from pinned host memory, refined records back
    hc = torch.from_numpy(np.ascontiguousarray(top).view(np.int32).reshape(-1, 7)).pin_memory()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        dc = hc.to(dev, non_blocking=True)
        rec = plan.refine(dc, steps=REFINE_STEPS, optimizer=args.optimizer)
    te = (time.perf_counter() - t0) / args.steps
    if rank != 0:
        return
    # algorithmic work per sample of the plain definition: the bilinear
    # sample (4 FMA) and its two slopes dB/dX, dB/dY (2 subtractions, a
    # product and an FMA each) weighted by g into their sums (1 FMA each)
    ops_per_sample = 14.0
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    max_mhz = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak_t = props.multi_processor_count * 128 * max_mhz * 1e6 / 1e12
    achieved = ops_per_sample * units / t_step / 1e12
    # algorithmic bytes: each evaluation reads, per candidate and frame, the
    # (64+1)^2 taps of its cutout footprint once (L2 serves overlapping
    # footprints, so this can exceed the copy bandwidth)
    esz = 4 if args.storage == "f32" else 2
    bytes_call = float(REFINE_N) * (REFINE_CUT + 1) ** 2 * esz * N * (REFINE_STEPS + 1)
    hbm = peaks.get("hbm_gbs", 6780.0)
    gbs = bytes_call / t_step / 1e9
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_t, "unit": "T FP32 ops/s",
            "frac": achieved / peak_t, "traffic": None, "work_per_unit": ops_per_sample,
            "kernel": "refine (bilinear cutout forward + adjoint, Adam)",
            "launches_per_step": 1, "avg_launch_ms": t_step * 1e3,
            "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {max_mhz:.0f} MHz",
            "footprint_gbs": gbs, "footprint_frac_of_hbm": gbs / hbm,
            "bytes_per_call": bytes_call}
    cfg = dict(config, candidates=REFINE_N, cutout=REFINE_CUT, steps=REFINE_STEPS,
               optimizer=args.optimizer, frames=N, storage=args.storage)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        import io
        import contextlib
        buf = io.StringIO()
        a2 = argparse.Namespace(**vars(args))
        a2.warmup, a2.steps = 0, 1
        with contextlib.redirect_stdout(buf):
            refine_reference(a2, d, config)
        r = json.loads(buf.getvalue())
        cpu = r["cpu_baseline"]
    snr_gain = float(np.median(rec["snr"] / np.maximum(top["snr"], 1e-6)))
    line = {
        "metric": REFINE_METRIC, "value": value, "unit": "G samples/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": cfg, "roofline": roof, "cpu_baseline": cpu,
        "clocks": clk, "median_snr_gain": snr_gain,
        "e2e": {"value": units * world / te / 1e9, "unit": "G samples/s",
                "h2d_bytes_per_step": int(hc.numel() * 4),
                "d2h_bytes_per_step": int(REFINE_N * 32), "s_per_step": te},
        "gpu_launches": int(plan.last_launch_count()) * args.steps,
        "device": torch.cuda.get_device_properties(dev).name}
    print(json.dumps(line))
    plan.close()


FRONT_GROUP, FRONT_OVERLAP, FRONT_SUM = 50, 5, 13
FRONT_METRIC = "front-end GB/s (median star removal + sums of 13 + 2x2 binning, 2048x2048x256)"


def front_bytes(N, H, W, groups):
    """Algorithmic bytes of one front-end pass: each kernel reads its input
    once and writes its output once (FP32)."""
    P = H * W
    med = sum(2 * (e - s) * P * 4 for s, e in groups)
    M = N // FRONT_SUM
    sums = (M * FRONT_SUM + M) * P * 4
    binb = N * P * 4 + N * (H // 2) * (W // 2) * 4
    return med, sums, binb


def front_reference(args, d, config):
    """The front-end oracle (numpy) on a bounded crop of the same frames."""
    from oracle import front
    fr = d["frames"]
    N = fr.shape[0]
    c = 64
    crop = np.ascontiguousarray(fr[:, :c, :c])
    t0 = time.perf_counter()
    front.median_subtract(crop[:FRONT_GROUP])
    front.sum_frames(crop, d["times"], FRONT_SUM)
    front.bin2x2(crop)
    el = time.perf_counter() - t0
    med, sums, binb = front_bytes(N, c, c, [(0, FRONT_GROUP)])
    v = (med + sums + binb) / el / 1e9
    sample = f"one group of {FRONT_GROUP} frames, sums and binning of a {c}x{c} crop, numpy oracle"
    print(json.dumps({
        "impl": "reference", "metric": FRONT_METRIC, "value": v, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config,
        "cpu_baseline": {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def bench_front(args, d, config, dev, world, rank, local):
    """The pre-tracking front end on the headline cube: one step = median
    removal over overlapping groups, the sums of every 13 frames and the
    2x2-binned cube, each kernel timed with CUDA events on the stream."""
    import torch
    import paper_2303_07293_gb300 as st
    from paper_2303_07293_gb300 import groups as grp
    N, H, W = d["frames"].shape
    stream = torch.cuda.current_stream(dev)
    frames = torch.from_numpy(d["frames"]).to(dev)
    out = torch.empty_like(frames)
    gr = grp.group_ranges(N, FRONT_GROUP, FRONT_OVERLAP)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def step():
        ev[0].record(stream)
        for s_, e_ in gr:
            st.median_subtract(frames[s_:e_], out=out[s_:e_], stream=stream)
        ev[1].record(stream)
        sums, _ = st.sum_frames(frames, d["times"], FRONT_SUM, stream=stream)
        ev[2].record(stream)
        binned = st.bin2x2(frames, stream=stream)
        ev[3].record(stream)
        return sums, binned

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    tm = [0.0, 0.0, 0.0]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
        torch.cuda.synchronize()
        for k in range(3):
            tm[k] += ev[k].elapsed_time(ev[k + 1]) / 1e3
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_step = e0.elapsed_time(e1) / 1e3 / args.steps
    med_b, sum_b, bin_b = front_bytes(N, H, W, gr)
    total = med_b + sum_b + bin_b
    if rank != 0:
        return
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6780.0)
    gbs = [b / (t / args.steps) / 1e9 for b, t in zip((med_b, sum_b, bin_b), tm)]
    roof = {"bound": "hbm", "achieved": gbs[0], "peak": hbm, "unit": "GB/s",
            "frac": gbs[0] / hbm, "traffic": None, "kernel": "k_median_subtract",
            "launches_per_step": len(gr), "avg_launch_ms": tm[0] / args.steps / len(gr) * 1e3,
            "peak_basis": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)",
            "per_kernel_gbs": {"median_subtract": gbs[0], "sum_frames": gbs[1], "bin2x2": gbs[2]},
            "per_kernel_frac": {"median_subtract": gbs[0] / hbm, "sum_frames": gbs[1] / hbm,
                                "bin2x2": gbs[2] / hbm}}
    cfg = dict(config, groups=[list(g) for g in gr], sum_every=FRONT_SUM)
    cpu = None
    if not args.no_cpu_baseline:
        import io
        import contextlib
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            front_reference(args, d, config)
        cpu = json.loads(buf.getvalue())["cpu_baseline"]
    print(json.dumps({
        "metric": FRONT_METRIC, "value": total / t_step / 1e9, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
        "roofline": roof, "cpu_baseline": cpu, "clocks": clk, "e2e": None,
        "gpu_launches": (len(gr) + 2) * args.steps,
        "device": torch.cuda.get_device_properties(dev).name}))


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = WORKLOADS[args.workload]
    d, batch_total = field_for(args, rank, world)
    ds = d if isinstance(d, list) else [d]
    d = ds[0]
    f = d["field"]
    N, H, W = d["frames"].shape
    adds = sum(float(x["frames"].size) * x["field"]["nvx"] * x["field"]["nvy"] for x in ds)
    # work of the whole job: the batch's total, or one field per rank
    job_adds = batch_total if batch_total is not None else adds * world
    scaling = "strong" if batch_total is not None else "weak"
    desc = wl["desc"]
    if any(v is not None for v in (args.width, args.frames, args.nv)):
        desc += f" -- resized: {W}x{H}x{N}, {f['nvx']}x{f['nvy']} grid"
    config = {"workload": f"{args.workload}: {desc}", "frames": N, "height": H, "width": W,
              "nv": [f["nvx"], f["nvy"]], "storage": args.storage, "shift": args.mode,
              "normalize": bool(args.normalize), "cr_clip": args.cr_clip, "tau": f["snr_threshold"],
              "tile": args.tile, "graph": bool(args.graph), "l2": l2_statement(ds, args.storage)}
    if batch_total is not None:
        config.update({"fields": BATCH, "fields_this_rank": len(ds),
                       "frames": [x["frames"].shape[0] for x in ds],
                       "sizes": [x["frames"].shape[1] for x in ds],
                       "nv": [x["field"]["nvx"] for x in ds], "adds_per_step": batch_total})

    if args.impl == "reference":
        if rank != 0:
            return
        if world > 1:
            # rank 0 runs alone (the other ranks have returned): give the
            # oracle the host's cores, which the launcher limited to one
            import oracle
            oracle.set_num_threads(len(os.sched_getaffinity(0)))
        if args.workload == "refine":
            return refine_reference(args, d, config)
        if args.workload == "front":
            return front_reference(args, d, config)
        unit = "G samples/s" if args.mode == "bilinear" else "G adds/s"
        rate, cores, sample, el = oracle_baseline(d, max(1.0, args.cpu_seconds / 3), args.mode)
        times = []
        for s in range(args.warmup + args.steps):
            r, cores, sample, el = oracle_baseline(d, max(1.0, args.cpu_seconds / 3), args.mode)
            if s >= args.warmup:
                times.append(r)
        v = float(np.median(times)) / 1e9
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": unit,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config,
            "cpu_baseline": {"value": v, "unit": unit, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2303_07293_gb300 as st
    if args.workload == "refine":
        return bench_refine(args, d, config, dev, world, rank, local)
    if args.workload == "front":
        return bench_front(args, d, config, dev, world, rank, local)

    frames = [torch.from_numpy(x["frames"]).to(dev) for x in ds]
    times = [x["times"] for x in ds]
    stream = torch.cuda.current_stream(dev)
    plan = st.Plan([x["field"] for x in ds], storage=args.storage, mode=args.mode,
                   normalize=bool(args.normalize), cr_clip=args.cr_clip if args.normalize else 0.0,
                   tile=args.tile, use_graph=bool(args.graph),
                   pending_capacity=(1 << 27) if batch_total is not None else (1 << 24),
                   stream=stream)
    cap = (1 << 24) if batch_total is not None else (1 << 22)
    out = torch.empty((cap, 7), dtype=torch.int32, device=dev)

    def step():
        nonlocal cap, out
        _, n, status = plan.search(frames, times, capacity=cap, out=out)
        if status == st.ST_ERR_OVERFLOW and n > cap:
            # more candidates than the buffer: grow it (the warm-up absorbs this)
            cap = int(n * 1.25)
            out = torch.empty((cap, 7), dtype=torch.int32, device=dev)
            _, n, status = plan.search(frames, times, capacity=cap, out=out)
        if status != st.ST_OK:
            raise RuntimeError(f"search status {status}")
        return n

    # warm-up (the first step autotunes); the wall-clock guard keeps the run
    # inside --time-budget: it stops warming up after 3 steps, then cuts the
    # timed steps, when the measured step time says the rest would not fit
    steps_requested, warmup_requested = args.steps, args.warmup
    t_w = 0.0
    done_w = 0
    for w_i in range(args.warmup):
        t0 = time.perf_counter()
        n_found = step()
        torch.cuda.synchronize()
        t_w = time.perf_counter() - t0
        done_w += 1
        extra = (args.e2e_steps * 1.2 * t_w if not args.no_e2e else 0.0) + \
            (args.cpu_seconds * 2 + 10 if not args.no_cpu_baseline else 0.0) + 30.0
        left = args.time_budget - (time.perf_counter() - T_START)
        if done_w >= 3 and (args.warmup - done_w + args.steps) * t_w + extra > left:
            break
    args.warmup = done_w
    if t_w > 0:
        left = args.time_budget - (time.perf_counter() - T_START) - extra
        fit = int(left // (t_w * 1.02))
        if world > 1:
            tt = torch.tensor([fit], device=dev)
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MIN)
            fit = int(tt.item())
        args.steps = max(1, min(args.steps, fit))
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stack_ms, stack_launch, launches = 0.0, 0, 0
    for _ in range(args.steps):
        n_found = step()
        ms, nl = plan.last_stack_kernel_time()
        stack_ms += ms
        stack_launch += nl
        launches += plan.last_launch_count()
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    t_step = ev0.elapsed_time(ev1) / 1e3 / args.steps
    if world > 1:
        tt = torch.tensor([t_step], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_step = float(tt.item())
    value = job_adds / t_step / 1e9

    # end to end through the host-buffer entry point (pinned frames)
    e2e = None
    if not args.no_e2e:
        hframes = [torch.from_numpy(x["frames"]).pin_memory() for x in ds]
        hbuf = np.zeros(cap, st.CAND_DTYPE)
        import ctypes as C
        fptr = (C.c_void_p * len(ds))(*[h.data_ptr() for h in hframes])
        tarr = [np.ascontiguousarray(t_, np.float64) for t_ in times]
        tptr = (C.c_void_p * len(ds))(*[t_.ctypes.data for t_ in tarr])
        cnt = C.c_int64()

        def host_step():
            s = st.lib().st_stack_search_host(plan._h, C.cast(fptr, C.c_void_p),
                                              C.cast(tptr, C.c_void_p),
                                              hbuf.ctypes.data_as(C.c_void_p), cap,
                                              C.byref(cnt))
            if s != st.ST_OK:
                raise RuntimeError(st.lib().st_last_error().decode())
            return cnt.value

        if world > 1:
            torch.distributed.barrier()
        n_e2e = max(1, args.e2e_steps)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            nh = host_step()
        te = (time.perf_counter() - t0) / n_e2e
        if world > 1:
            tt = torch.tensor([te], device=dev)
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            te = float(tt.item())
        e2e = {"value": job_adds / te / 1e9, "unit": "G adds/s",
               "h2d_bytes_per_step": int(sum(h.numel() * 4 for h in hframes) +
                                         sum(t_.nbytes for t_ in tarr)),
               "d2h_bytes_per_step": int(nh * 28 + 32), "s_per_step": te, "steps": n_e2e}

    if rank != 0:
        return
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks = measured_peaks()
    max_mhz = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak_t = sms * 128 * max_mhz * 1e6 / 1e12  # FP32 adds (or FMAs) per second, T
    stack_avg_ms = stack_ms / max(stack_launch, 1)
    variant = plan.stack_variant_name(0)
    config["stack_variant"] = variant
    tr = STACK_TRAFFIC.get((args.workload, args.storage, args.mode, variant))
    traffic = tr[0] if tr and tr[1] == stack_source_sha() and stack_launch == args.steps \
        and (args.width, args.frames, args.nv) == (None, None, None) else None
    if traffic is not None:
        traffic_note = "DRAM bytes of one launch from the stored ncu capture of this code"
    elif tr is None:
        traffic_note = (f"null: no ncu DRAM capture stored for this workload and variant "
                        f"({variant})")
    elif tr[1] != stack_source_sha():
        traffic_note = (f"null: the stored capture ({tr[0] / 1e9:.2f} GB per launch) was taken "
                        f"on k_stack_fast.cu code {tr[1]}, the kernel is now "
                        f"{stack_source_sha()}")
    else:
        traffic_note = "null: the stored capture is of one launch per step"
    # algorithmic work per pixel*frame*velocity: 1 add (nearest), 4 FMA (bilinear)
    per_unit = 4.0 if args.mode == "bilinear" else 1.0
    achieved = per_unit * adds / (stack_ms / 1e3 / args.steps) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_t,
            "unit": "T FMA/s" if args.mode == "bilinear" else "T adds/s",
            "frac": achieved / peak_t, "traffic": traffic, "traffic_note": traffic_note,
            "work_per_unit": per_unit,
            "kernel": "stack (shift-and-stack + threshold)", "launches_per_step":
                stack_launch / args.steps, "avg_launch_ms": stack_avg_ms,
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x {max_mhz:.0f} MHz (max SM clock)"}
    if clk and clk.get("sm_mhz"):
        roof["frac_at_observed_clock"] = achieved / (sms * 128 * clk["sm_mhz"] * 1e6 / 1e12)
    unit = "G samples/s" if args.mode == "bilinear" else "G adds/s"
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, cores, sample, el = oracle_baseline(d, args.cpu_seconds, args.mode)
        cpu = {"value": rate / 1e9, "unit": unit, "cores": cores, "kind": "oracle",
               "sample": sample, "seconds": el}
    if e2e:
        e2e["unit"] = unit
    if args.graph:
        config["graph_replayed"] = plan.last_graph_replayed()
    tracks = None
    if args.tracks:
        tt0 = torch.cuda.Event(enable_timing=True)
        tt1 = torch.cuda.Event(enable_timing=True)
        plan.link_tracks(out[:min(n_found, cap)], min(n_found, cap))   # warm-up
        tt0.record(stream)
        trk = plan.link_tracks(out[:min(n_found, cap)], min(n_found, cap))
        tt1.record(stream)
        torch.cuda.synchronize()
        tracks = {"detections": int(min(n_found, cap)), "tracks": int(len(trk)),
                  "link_ms": tt0.elapsed_time(tt1), "r_xy": 2, "r_v": 1}
    precision = None
    if args.precision and batch_total is None:
        cand = out[:min(n_found, cap)].cpu().numpy().view(st.CAND_DTYPE).reshape(-1)
        precision = precision_report(args, d, cand)
    line = {
        "metric": METRIC, "value": value, "unit": unit, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
        "higher_is_better": True, "scaling": scaling, "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config,
        "fields_per_hr": 3600.0 / t_step * (BATCH if batch_total is not None else world),
        "candidates": int(n_found), "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
        "e2e": e2e, "gpu_launches": int(launches), "device": props.name}
    if (args.steps, args.warmup) != (steps_requested, warmup_requested):
        line["time_guard"] = {"steps_requested": steps_requested,
                              "warmup_requested": warmup_requested,
                              "budget_s": args.time_budget, "warmup_step_s": t_w}
    if precision:
        line["precision"] = precision
    if tracks:
        line["tracks"] = tracks
    print(json.dumps(line))
    plan.close()


if __name__ == "__main__":
    main()
