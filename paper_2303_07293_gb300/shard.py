"""Host-side sharding of a multi-field search over replicas (one process per GPU).

The search has no exchange step (every field, and every velocity of a field,
is independent: Sec. 2.1 searches each trial motion on its own), so N GPUs
run N independent plans.  This module holds the host logic around them:

* ``assign_fields`` — longest-processing-time-first assignment of fields to
  ranks by their work P*N*N_v, so the ranks finish close together;
* ``merge_candidates`` — concatenation of per-rank candidate lists (with the
  field indices mapped back to the global numbering) and the library's
  deterministic (field, k, y, x) order, so the merged list equals the one a
  single plan over every field returns;
* ``gather_candidates`` — the per-rank lists collected on rank 0 through
  ``torch.distributed`` (any backend; gloo on CPU in the tests).

No collective runs on the data path: only the final variable-length lists
move, once.
"""
import numpy as np

from . import CAND_DTYPE


def field_work(field):
    """Naive pixel*frame*velocity count of a field (its stack work)."""
    return (int(field["width"]) * int(field["height"]) * int(field["n_frames"]) *
            int(field["nvx"]) * int(field["nvy"]))


def assign_fields(fields, world):
    """Field indices per rank: longest work first, each to the least loaded
    rank (ties to the lower rank).  Deterministic."""
    order = sorted(range(len(fields)), key=lambda i: (-field_work(fields[i]), i))
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += field_work(fields[i])
    return [sorted(x) for x in out]


def merge_candidates(parts):
    """parts: list of (global field indices of the rank's plan, candidate
    array of that plan).  Returns one array in (field, k, y, x) order."""
    chunks = []
    for gidx, cand in parts:
        c = np.array(cand, dtype=CAND_DTYPE, copy=True)
        if len(c):
            c["field"] = np.asarray(gidx, np.int32)[c["field"]]
        chunks.append(c)
    allc = np.concatenate(chunks) if chunks else np.zeros(0, CAND_DTYPE)
    order = np.lexsort((allc["x"], allc["y"], allc["k"], allc["field"]))
    return allc[order]


def gather_candidates(gidx, cand, group=None):
    """Collects every rank's (field indices, candidates) on rank 0 and returns
    the merged list there (None on the other ranks)."""
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    payload = (list(map(int, gidx)), np.ascontiguousarray(cand, dtype=CAND_DTYPE).tobytes())
    got = [None] * world if rank == 0 else None
    dist.gather_object(payload, got, dst=0, group=group)
    if rank != 0:
        return None
    parts = [(g, np.frombuffer(b, dtype=CAND_DTYPE)) for g, b in got]
    return merge_candidates(parts)
