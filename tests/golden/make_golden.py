"""Writes the stored expected values under tests/golden/ by calling only the
CPU oracle (oracle/).  Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import OracleProblem  # noqa: E402


def main():
    # 16^3, 4 levels, b = A * ones, x0 = 0, 50 iterations, no tolerance stop:
    # the small plain-FP64 workload.
    p = OracleProblem(16, 16, 16, levels=4)
    x, hist = p.pcg(p.rhs(), max_iters=50, tol=0.0)
    with open(os.path.join(HERE, "pcg_history_16cubed.txt"), "w") as f:
        f.write("# relative residual ||r_k||/||r_0|| of FP64 MG-PCG, 16^3, 4 levels, b = A*ones, x0 = 0\n")
        f.write("# written by tests/golden/make_golden.py from the CPU oracle\n")
        for h in hist:
            f.write("%.17e\n" % h)
    # level sizes and nonzero counts of the 192^3 hierarchy from the closed
    # form (3nx-2)(3ny-2)(3nz-2); cross-checked against the oracle's CRS at
    # the small sizes by tests/test_oracle_operator.py
    with open(os.path.join(HERE, "hierarchy_192cubed.txt"), "w") as f:
        f.write("# level nx ny nz n nnz  (closed form)\n")
        for l in range(4):
            s = 192 >> l
            f.write("%d %d %d %d %d %d\n" % (l, s, s, s, s ** 3, (3 * s - 2) ** 3))


if __name__ == "__main__":
    main()
