"""Host policy that turns per-tile variance into render counts (Sec. 4.1.1)."""

import numpy as np
import pytest

from paper_2305_07083_gb300 import adaptive


def test_redundancy_bounds_and_monotone():
    rng = np.random.default_rng(0)
    v = rng.random(100) ** 3
    k = adaptive.redundancy(v, 1, 6)
    assert k.min() == 1 and k.max() <= 6
    order = np.argsort(v)
    assert (np.diff(k[order]) >= 0).all()          # more variance, never fewer renders
    assert (k[v <= np.median(v)] == 1).all()


def test_redundancy_edge_cases():
    assert (adaptive.redundancy(np.zeros(5), 2, 4) == 2).all()
    k = adaptive.redundancy(np.array([0.0, 0.0, 0.0, 1.0, np.nan]), 1, 5)
    assert list(k) == [1, 1, 1, 5, 1]
    with pytest.raises(ValueError):
        adaptive.redundancy(np.ones(3), 0, 4)
