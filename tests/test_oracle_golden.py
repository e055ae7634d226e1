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


def test_hierarchy_192cubed_fixture_matches_closed_form_counts():
    # rows n_l = m^3 and nonzeros (3m - 2)^3 of an m^3 grid, m = 192 / 2^l
    rows = np.loadtxt(os.path.join(HERE, "hierarchy_192cubed.txt"), dtype=np.int64)
    m = [192 >> l for l in range(4)]
    assert list(rows[:, 4]) == [v ** 3 for v in m] == [7077888, 884736, 110592, 13824]
    assert list(rows[:, 5]) == [(3 * v - 2) ** 3 for v in m] == [189119224, 23393656, 2863288, 343000]
