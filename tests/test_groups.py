"""Host logic of the frame groups (paper_2303_07293_gb300/groups.py) against
the pinned front-end oracle's group rule, over a sweep of sizes and
overlaps; and the invariants a caller relies on (full coverage, the stated
overlap, every group the same size)."""
import itertools

import pytest

from oracle import front
from paper_2303_07293_gb300 import groups


def test_group_ranges_equal_oracle_and_cover_the_sequence():
    for n, size, ov in itertools.product([1, 7, 49, 50, 51, 100, 256, 1000], [5, 13, 50, 64],
                                         [0, 1, 4]):
        if ov >= size:
            continue
        got = groups.group_ranges(n, size, ov)
        assert got == front.group_ranges(n, size, ov), (n, size, ov)
        covered = set()
        for s, e in got:
            covered.update(range(s, e))
            assert e - s == min(size, n)
        assert covered == set(range(n))
        for (s0, e0), (s1, e1) in zip(got, got[1:]):
            assert s1 <= e0 - ov                      # consecutive groups share >= ov frames


def test_group_size_equal_oracle():
    for field_px, v, cad in itertools.product([512, 1024, 2048], [1.0, 7.5, 100.0, 1000.0],
                                              [25 / 3600, 50 / 3600, 0.1]):
        assert groups.group_size(field_px, v, cad) == front.group_size(field_px, v, cad)


def test_overlap_must_be_smaller_than_the_group():
    with pytest.raises(ValueError):
        groups.group_ranges(100, 10, 10)
