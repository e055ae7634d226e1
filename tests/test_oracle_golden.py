"""Regression pin: the oracle's 16^3 residual history against the stored
fixture written by tests/golden/make_golden.py (oracle only)."""
import os

import numpy as np

from oracle import OracleProblem

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_history_16cubed_fixture():
    ref = np.loadtxt(os.path.join(HERE, "pcg_history_16cubed.txt"))
    p = OracleProblem(16, 16, 16, levels=4)
    _, hist = p.pcg(p.rhs(), max_iters=50, tol=0.0)
    np.testing.assert_array_equal(hist, ref)


def test_hierarchy_192cubed_fixture_matches_survey_counts():
    rows = np.loadtxt(os.path.join(HERE, "hierarchy_192cubed.txt"), dtype=np.int64)
    assert list(rows[:, 4]) == [7077888, 884736, 110592, 13824]
    assert list(rows[:, 5]) == [189119224, 23393656, 2863288, 343000]
