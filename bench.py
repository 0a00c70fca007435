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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "speculoos": dict(name="speculoos", desc="2048x2048x256, 801x801 velocity grid"),
    "mid": dict(name="mid", desc="1024x1024x64, 161x161 velocity grid"),
    "tiny": dict(name="tiny", desc="128x128x16, 21x21 velocity grid"),
    "batched": dict(name="batched", desc="24 fields: N in [40,400], sizes {512,1024,2048}^2, "
                    "baselines 1-8 h, grid step 1 px/baseline, +-60 px/h, one plan"),
}
METRIC = "G pixel*frame*velocity adds/s (2048x2048x256, 801x801 grid)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="speculoos", choices=list(WORKLOADS))
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--mode", default="nearest", choices=["nearest", "bilinear"])
    ap.add_argument("--normalize", type=int, default=1)
    ap.add_argument("--cr-clip", type=float, default=10.0,
                    help="zero |I| > cr_clip sigma after normalisation (cosmic-ray removal)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tile", type=int, default=-1,
                    help="-1 autotune (first warm-up step), 0 default, 1 direct-gather, 2.. variant")
    return ap.parse_args()


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


def oracle_baseline(d, seconds, rank0=True):
    """Oracle (FP32-sequential, as it stands) on a slab of velocity planes of
    the same field; returns (adds/s, cores, sample description, elapsed)."""
    import oracle
    oracle.lib()  # build/load outside the timed region
    f = d["field"]
    N, H, W = d["frames"].shape
    cores = oracle.num_threads()
    fr = np.nan_to_num(d["frames"], nan=0.0)
    nk = f["nvx"] * f["nvy"]
    k0 = nk // 2 - cores // 2
    t0 = time.perf_counter()
    oracle.search(fr, d["times"], f, prec="fp32", k_begin=k0, k_end=k0 + cores)
    dt = time.perf_counter() - t0
    per_round = dt
    rounds = max(1, int(seconds / max(per_round, 1e-3)) - 1)
    k1 = min(nk, k0 + cores + rounds * cores)
    t0 = time.perf_counter()
    oracle.search(fr, d["times"], f, prec="fp32", k_begin=k0 + cores, k_end=k1)
    el = time.perf_counter() - t0
    n_planes = k1 - (k0 + cores)
    adds = float(W * H * N) * n_planes
    return adds / el, cores, (f"{n_planes} velocity planes (k {k0 + cores}..{k1 - 1}) of the "
                              f"full {W}x{H}x{N} field, FP32-sequential oracle"), el


def field_for(args, rank):
    import synth
    w = WORKLOADS[args.workload]["name"]
    seed = synth.BASE_SEED + {"tiny": 1, "mid": 2, "speculoos": 3, "batched": 4}[w] + 100000 * rank
    if w == "batched":
        return [synth.make_field(w, seed=seed, index=j) for j in range(24)]
    return synth.make_field(w, seed=seed)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = WORKLOADS[args.workload]
    d = field_for(args, rank)
    ds = d if isinstance(d, list) else [d]
    d = ds[0]
    f = d["field"]
    N, H, W = d["frames"].shape
    adds = sum(float(x["frames"].size) * x["field"]["nvx"] * x["field"]["nvy"] for x in ds)
    config = {"workload": f"{args.workload}: {wl['desc']}", "frames": N, "height": H, "width": W,
              "nv": [f["nvx"], f["nvy"]], "storage": args.storage, "shift": args.mode,
              "normalize": bool(args.normalize), "cr_clip": args.cr_clip, "tau": f["snr_threshold"],
              "tile": args.tile, "l2": "inputs larger than L2 (frame cube > 129 MB)"}
    if len(ds) > 1:
        config.update({"fields": len(ds), "frames": [x["frames"].shape[0] for x in ds],
                       "sizes": [x["frames"].shape[1] for x in ds],
                       "nv": [x["field"]["nvx"] for x in ds], "adds_per_step": adds})

    if args.impl == "reference":
        if rank != 0:
            return
        rate, cores, sample, el = oracle_baseline(d, max(1.0, args.cpu_seconds / 3))
        times = []
        for s in range(args.warmup + args.steps):
            r, cores, sample, el = oracle_baseline(d, max(1.0, args.cpu_seconds / 3))
            if s >= args.warmup:
                times.append(r)
        v = float(np.median(times)) / 1e9
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": "G adds/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config,
            "cpu_baseline": {"value": v, "unit": "G adds/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "G adds/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2303_07293_gb300 as st

    frames = [torch.from_numpy(x["frames"]).to(dev) for x in ds]
    times = [x["times"] for x in ds]
    stream = torch.cuda.current_stream(dev)
    plan = st.Plan([x["field"] for x in ds], storage=args.storage, mode=args.mode, normalize=bool(args.normalize),
                   cr_clip=args.cr_clip if args.normalize else 0.0, tile=args.tile,
                   pending_capacity=1 << 24, stream=stream)
    cap = 1 << 22
    out = torch.empty((cap, 7), dtype=torch.int32, device=dev)

    def step():
        _, n, status = plan.search(frames, times, capacity=cap, out=out)
        if status != st.ST_OK:
            raise RuntimeError(f"search status {status}")
        return n

    for _ in range(args.warmup):
        n_found = step()
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
    value = adds * world / t_step / 1e9

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
        t0 = time.perf_counter()
        for _ in range(args.steps):
            nh = host_step()
        te = (time.perf_counter() - t0) / args.steps
        if world > 1:
            tt = torch.tensor([te], device=dev)
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            te = float(tt.item())
        e2e = {"value": adds * world / te / 1e9, "unit": "G adds/s",
               "h2d_bytes_per_step": int(sum(h.numel() * 4 for h in hframes) +
                                         sum(t_.nbytes for t_ in tarr)),
               "d2h_bytes_per_step": int(nh * 28 + 32), "s_per_step": te}

    if rank != 0:
        return
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks = measured_peaks()
    max_mhz = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak_t = sms * 128 * max_mhz * 1e6 / 1e12  # FP32 adds per second, T
    stack_avg_ms = stack_ms / max(stack_launch, 1)
    achieved = adds / (stack_ms / 1e3 / args.steps) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_t, "unit": "T adds/s",
            "frac": achieved / peak_t, "traffic": None,
            "kernel": "stack (shift-and-stack + threshold)", "launches_per_step":
                stack_launch / args.steps, "avg_launch_ms": stack_avg_ms,
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x {max_mhz:.0f} MHz (max SM clock)"}
    if clk and clk.get("sm_mhz"):
        roof["frac_at_observed_clock"] = achieved / (sms * 128 * clk["sm_mhz"] * 1e6 / 1e12)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, cores, sample, el = oracle_baseline(d, args.cpu_seconds)
        cpu = {"value": rate / 1e9, "unit": "G adds/s", "cores": cores, "kind": "oracle",
               "sample": sample, "seconds": el}
    line = {
        "metric": METRIC, "value": value, "unit": "G adds/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config, "fields_per_hr": 3600.0 / t_step * world,
        "candidates": int(n_found), "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
        "e2e": e2e, "gpu_launches": int(launches), "device": props.name}
    print(json.dumps(line))
    plan.close()


if __name__ == "__main__":
    main()
