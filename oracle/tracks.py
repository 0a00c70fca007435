"""Oracle of the linking of detections into tracks (test infrastructure only).

Only the tests and ``bench.py``'s CPU-baseline leg may import this module.
The search reports per-velocity local maxima (Sec. 2.1); one moving object
yields detections at neighbouring trial velocities and positions.  The paper
returns tracks "with corresponding speed, PA, pixel coordinates and S/N"
(Sec. 2.1) and gives no linking rule; the reading here:

* two detections of the same field are linked when their pixels differ by
  at most r_xy in x and in y and their velocity indices by at most r_v in a
  and in b; a track is a connected component of the links;
* a track is represented by its detection of highest S/N (ties: the first in
  the (field, k, y, x) order), reported with the component's size;
* velocity (vx, vy) from the grid; speed = hypot(vx, vy) in FP64; PA in
  degrees in [0, 360), measured from the image's -y axis towards its -x
  axis (north up, east left), atan2(-vx, -vy) in FP64;
* tracks are listed in the order of their first detection in (field, k, y, x).
"""
import math

import numpy as np


def link_tracks(cand, grids, r_xy=2, r_v=1):
    """cand: structured array (x, y, k, field, stack, snr, n_cov) sorted by
    (field, k, y, x); grids: per field (vx0, dvx, nvx, vy0, dvy, nvy).
    Returns a list of dicts, one per track."""
    n = len(cand)
    parent = list(range(n))

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i

    def unite(i, j):
        ri, rj = find(i), find(j)
        if ri != rj:
            parent[max(ri, rj)] = min(ri, rj)

    # detections by (field, a, b) for the neighbour search
    cells = {}
    for i in range(n):
        f = int(cand["field"][i])
        nvx = grids[f][2]
        k = int(cand["k"][i])
        cells.setdefault((f, k % nvx, k // nvx), []).append(i)
    for i in range(n):
        f = int(cand["field"][i])
        nvx = grids[f][2]
        k = int(cand["k"][i])
        a, b = k % nvx, k // nvx
        x, y = int(cand["x"][i]), int(cand["y"][i])
        for da in range(-r_v, r_v + 1):
            for db in range(-r_v, r_v + 1):
                for j in cells.get((f, a + da, b + db), ()):
                    if j > i and abs(int(cand["x"][j]) - x) <= r_xy and \
                            abs(int(cand["y"][j]) - y) <= r_xy:
                        unite(i, j)
    members = {}
    for i in range(n):
        members.setdefault(find(i), []).append(i)
    out = []
    for root in sorted(members):
        idx = members[root]
        best = idx[0]
        for i in idx[1:]:
            if cand["snr"][i] > cand["snr"][best]:
                best = i
        f = int(cand["field"][best])
        vx0, dvx, nvx, vy0, dvy, nvy = grids[f]
        k = int(cand["k"][best])
        vx = vx0 + (k % nvx) * dvx
        vy = vy0 + (k // nvx) * dvy
        pa = math.degrees(math.atan2(-vx, -vy)) % 360.0
        out.append(dict(x=int(cand["x"][best]), y=int(cand["y"][best]), k=k, field=f,
                        stack=float(cand["stack"][best]), snr=float(cand["snr"][best]),
                        n_cov=int(cand["n_cov"][best]), members=len(idx), vx=vx, vy=vy,
                        speed=math.hypot(vx, vy), pa=pa))
    return out
