"""The bench's dual-tree schedule (host logic, no GPU) against the oracle's rung rule.

Inside an interval of the fixed rung no particle of the fixed rungs may be active: they move on
straight lines there, which is what lets their tree be built once at the interval's middle.
The interval's boundaries, where they are active, get a full solve."""
import numpy as np
import pytest

import bench
from oracle import kdk


@pytest.mark.parametrize("max_rung,fixed", [(5, 0), (5, 2), (5, 3), (5, 4), (3, 1)])
def test_fixed_rungs_are_idle_inside_their_intervals(max_rung, fixed):
    m = 1 << (max_rung - fixed)
    base = 1 << max_rung
    seen = {}
    for t in range(1, 3 * base + 1):
        role, interval, to_mid = bench.dual_role(t, max_rung, fixed)
        s = t % base
        slow = np.arange(fixed + 1, dtype=np.uint8)
        fast = np.arange(fixed + 1, max_rung + 1, dtype=np.uint8)
        if role == "full":
            assert t % m == 0
            assert kdk.active(np.array([fixed], np.uint8), s, max_rung).all()
        else:
            assert not kdk.active(slow, s, max_rung).any()
            # the finest rung is active on every substep, dual or not
            assert kdk.active(fast[-1:], s, max_rung).all()
            # the drift target is the interval's middle, the same for all its substeps
            assert t + to_mid == interval * m + m / 2
            seen.setdefault(interval, set()).add(t)
    for interval, ts in seen.items():
        assert ts == set(range(interval * m + 1, interval * m + m)) & set(range(1, 3 * base + 1))
