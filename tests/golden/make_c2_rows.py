"""Write tests/golden/c2_3d_invr_n262144_rows.txt with the FP64 oracle only.

    python tests/golden/make_c2_rows.py      (single core, about half an hour)

Workload: 3D 1/r, N = 262144 points uniform in [-1, 1]^3 (seed 1002), one
N(0, 1) right-hand side (seed 2002), octree leaves of <= 64 points (kappa 4),
H2*(b+t) with eps = 1e-6.  For 1024 rows sampled with numpy default_rng(5)
it stores the oracle's compressed product (K~ q)_i and the exact (K q)_i.
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dense, h2  # noqa: E402
from paper_2309_14085_gb300 import inputs  # noqa: E402


def main():
    w = inputs.workload("c2_3d_invr_n262144")
    P, q = w["points"], w["q"]
    t0 = time.time()
    H = h2.H2(P, "invr", n_max=64, eps=1e-6, store_m2l=False)
    t1 = time.time()
    phi = H.matvec(q)
    t2 = time.time()
    rows = np.random.default_rng(5).choice(P.shape[0], 1024, replace=False)
    exact = dense.rows("invr", P, q, rows, chunk=16)
    re = dense.relative_error(phi[rows], exact)
    out = os.path.join(HERE, "c2_3d_invr_n262144_rows.txt")
    with open(out, "w") as f:
        f.write("# Oracle H2*(b+t) rows of K~ q and exact rows of K q for the 3D 1/r workload\n")
        f.write("# N = 262144 (points seed 1002, rhs seed 2002), leaf size 64, eps 1e-6; rows:\n")
        f.write("# numpy default_rng(5).choice(N, 1024, replace=False).  Written by\n")
        f.write("# tests/golden/make_c2_rows.py (oracle only): build %.0f s, MVP %.0f s,\n"
                % (t1 - t0, t2 - t1))
        f.write("# sampled relative error %.6e\n" % re)
        f.write("# columns: row  oracle_Ktilde_q  exact_K_q\n")
        for i, a, b in zip(rows, phi[rows], exact):
            f.write("%d %.17e %.17e\n" % (i, a, b))
    print(out, "RE", re)


if __name__ == "__main__":
    main()
