"""Host-side helpers of bench.py (no GPU): the algorithmic-work formulas the
bench lines divide by, the code hash that keeps a stored DRAM traffic figure
tied to the kernel it was measured on, and the precision / recovery report
(fed here with the oracle's own candidates, which must score exactly)."""
import argparse

import numpy as np

import bench
import oracle
import synth


def test_work_formulas():
    # refinement: candidates x cutout pixels x frames x (steps + 1) evaluations
    assert bench.refine_units(300) == 4096 * 64 * 64 * 300 * 21
    # front end: each kernel reads its input once and writes its output once
    med, sums, binb = bench.front_bytes(256, 2048, 2048, [(0, 50), (45, 95)])
    P = 2048 * 2048
    assert med == 2 * (50 + 50) * P * 4
    assert sums == (19 * 13 + 19) * P * 4            # 19 sums of 13 frames
    assert binb == 256 * P * 4 + 256 * 1024 * 1024 * 4


def test_code_hash_ignores_comments_only():
    h = bench.stack_source_sha()
    assert len(h) == 12 and h == bench.stack_source_sha()


def test_precision_report_on_oracle_candidates():
    from paper_2303_07293_gb300 import CAND_DTYPE
    d = synth.make_field("tiny", seed=synth.BASE_SEED + 1)
    r = oracle.search(np.nan_to_num(d["frames"]), d["times"], d["field"], prec="fp32")
    c = np.zeros(len(r), CAND_DTYPE)
    for k in ("x", "y", "k", "n_cov"):
        c[k] = r[k]
    c["stack"] = r["stack"]
    c["snr"] = r["snr"]
    args = argparse.Namespace(normalize=0, cr_clip=0.0, mode="nearest", storage="f32")
    rep = bench.precision_report(args, d, c)
    assert rep["points"] == len(c) and rep["err_max_rel"] < 1e-6
    assert rep["recovered"] == rep["movers"] == 3


def test_l2_statement_follows_the_stored_cube():
    class Cube:  # only the element count matters
        def __init__(self, n):
            self.size = n
    head = [{"frames": Cube(256 * 2048 * 2048)}]
    assert bench.l2_statement(head, "f32") == \
        "inputs larger than L2 (stored frame cube 4295 MB > 129 MB)"
    assert bench.l2_statement(head, "bf16").startswith("inputs larger than L2 (stored frame cube 2147")
    tiny = [{"frames": Cube(16 * 128 * 128)}]
    assert bench.l2_statement(tiny, "f16").startswith("inputs smaller than L2")


def test_reference_arm_prints_one_contract_line():
    # the reference arm (the CPU oracle) runs without a GPU: one JSON line
    # with the keys of the benchmark contract, its own baseline and e2e
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--workload", "tiny", "--steps", "1", "--warmup", "0",
                        "--cpu-seconds", "1"], capture_output=True, text=True, timeout=600,
                       cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("tiny")
