"""Multi-process (replica) path on CPU: fields assigned to 2 gloo ranks, each
rank's candidate list gathered and merged on rank 0 must equal the list of a
single search over every field (the search has no exchange step, Sec. 2.1;
each rank's search is stood in for by the oracle here, which needs no GPU)."""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")


def _fields():
    out = []
    for j, (w, n, nv) in enumerate([(64, 12, 9), (96, 16, 11), (48, 10, 7), (80, 14, 13),
                                    (64, 9, 5)]):
        d = synth.make_field("tiny", seed=900 + j, width=w, n_frames=n, nv=nv)
        out.append(d)
    return out


def _cands(d, field_index):
    from paper_2303_07293_gb300 import CAND_DTYPE
    r = oracle.search(d["frames"], d["times"], d["field"], prec="fp32")
    c = np.zeros(len(r), CAND_DTYPE)
    for k in ("x", "y", "k", "n_cov"):
        c[k] = r[k]
    c["stack"] = r["stack"].astype(np.float32)
    c["snr"] = r["snr"].astype(np.float32)
    c["field"] = field_index
    return c


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    from paper_2303_07293_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ds = _fields()
    mine = shard.assign_fields([d["field"] for d in ds], world)[rank]
    # this rank's plan numbers its fields 0..len(mine)-1
    local = [_cands(ds[g], i) for i, g in enumerate(mine)]
    cand = np.concatenate(local) if local else np.zeros(0, dtype=_cands(ds[0], 0).dtype)
    merged = shard.gather_candidates(mine, cand)
    if rank == 0:
        np.save(out_path, merged)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_assign_fields_lpt():
    from paper_2303_07293_gb300 import shard
    fs = [dict(width=w, height=w, n_frames=n, nvx=v, nvy=v)
          for w, n, v in [(512, 40, 100), (2048, 300, 800), (1024, 100, 300), (512, 400, 50),
                          (2048, 60, 700), (1024, 250, 500)]]
    for world in (1, 2, 3, 4, 8):
        a = shard.assign_fields(fs, world)
        assert sorted(i for r in a for i in r) == list(range(len(fs)))
        loads = [sum(shard.field_work(fs[i]) for i in r) for r in a]
        # LPT bound: no rank exceeds the mean by more than the largest field
        assert max(loads) <= sum(loads) / world + max(map(shard.field_work, fs))
    assert shard.assign_fields(fs, 2) == shard.assign_fields(fs, 2)   # deterministic


def test_gloo_two_ranks_merge_equals_single_search():
    import torch.multiprocessing as mp
    from paper_2303_07293_gb300 import shard
    ds = _fields()
    single = shard.merge_candidates([(list(range(len(ds))),
                                      np.concatenate([_cands(d, i) for i, d in enumerate(ds)]))])
    assert len(single) > 0
    with tempfile.TemporaryDirectory() as tmp:
        out = os.path.join(tmp, "merged.npy")
        mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True,
                           start_method="spawn")
        merged = np.load(out)
    assert merged.tobytes() == single.tobytes()
    assert np.all(np.diff(merged["field"]) >= 0)
