"""Frame grouping of the fast-mover search (host logic; Sec. 2.1).

An object can only be detected if it is above threshold in at least half of
the frames searched together, so a long sequence is searched in slightly
overlapping groups, each short enough that the fastest searched object stays
in the field for the stated fraction (70 %) of the group's span.
"""
import math


def group_size(field_px, v_max, cadence, presence=0.7):
    """Frames per group: the group may span field_px / (presence * v_max)
    time units (v_max in px per time unit), i.e. that many cadences."""
    span = field_px / (presence * v_max)
    return max(1, int(math.floor(span / cadence)))


def group_ranges(n_frames, size, overlap):
    """[start, end) of consecutive groups of `size` frames sharing `overlap`
    frames; the last group is moved back to end at the last frame."""
    if size <= overlap:
        raise ValueError("overlap must be smaller than the group size")
    if n_frames <= size:
        return [(0, n_frames)]
    starts = list(range(0, n_frames - size, size - overlap))
    return [(s, s + size) for s in starts] + [(n_frames - size, n_frames)]
