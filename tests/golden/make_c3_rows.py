"""Write tests/golden/c3_2d_log_n1048576_rows.txt with the FP64 oracle only.

    python tests/golden/make_c3_rows.py        (single core, a few seconds)

Workload: 2D log r, N = 2^20 points uniform in [-1, 1]^2 (seed 1003), 64
N(0, 1) right-hand sides (seed 2003).  For 16 rows sampled with numpy
default_rng(7) it stores the exact rows of K Q (the dense definition), against
which the benchmark reports the relative error of its 64-RHS products.
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dense  # noqa: E402
from paper_2309_14085_gb300 import inputs  # noqa: E402


def main():
    w = inputs.workload("c3_2d_log_n1048576")
    P, Q = w["points"], w["q"].reshape(w["N"], w["nrhs"])
    rows = np.random.default_rng(7).choice(P.shape[0], 16, replace=False)
    exact = dense.rows("log2d", P, Q, rows)
    out = os.path.join(HERE, "c3_2d_log_n1048576_rows.txt")
    with open(out, "w") as f:
        f.write("# Exact rows of K Q for the 64-RHS workload (2D log r, N = 2^20, points seed\n")
        f.write("# 1003, right-hand sides seed 2003); rows numpy default_rng(7).choice(N, 16,\n")
        f.write("# replace=False).  Written by tests/golden/make_c3_rows.py (oracle only).\n")
        f.write("# columns: row, then (K Q)[row, 0 .. 63]\n")
        for i, r in zip(rows, exact):
            f.write("%d " % i + " ".join("%.17e" % v for v in r) + "\n")
    print(out)


if __name__ == "__main__":
    main()
