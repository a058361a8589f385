"""The library's host-side stopping criterion (fo_stop_check, Sec. 5.7) agrees with the
oracle's on hand-made and random histories (no GPU needed)."""
import numpy as np
import pytest

from oracle import ppl as oppl


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_05709_gb300 import api as a
    return a


def test_stop_check_matches_oracle(api):
    rng = np.random.default_rng(0)
    cases = [([10.0] * 25 + [1.0 + 1e-4 * k for k in range(20)], None),
             ([1.0 + 0.05 * k for k in range(45)], None),
             ([10.0] * 25 + [1.0] * 20, [1.005, 0.996]),
             ([10.0] * 25 + [1.0] * 20, [1.02]),
             ([5.0] * 40 + [1.0] * 11, None)]
    for _ in range(200):
        n = int(rng.integers(5, 60))
        vals = list(1.0 + np.cumsum(rng.normal(0, 10.0 ** rng.uniform(-5, -1), n)))
        C = None if rng.random() < 0.5 else list(1.0 + rng.normal(0, 10.0 ** rng.uniform(-4, -1), int(rng.integers(1, 5))))
        cases.append((vals, C))
    for vals, C in cases:
        for prev in (10, 11, 5):
            assert api.stop_check(vals, C, prev=prev) == oppl.stop_check(vals, C, prev=prev), (vals, C, prev)
