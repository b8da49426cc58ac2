"""Write tests/golden/oracle_re_paper_configs.txt with the FP64 oracle only.

    python tests/golden/make_paper_configs.py        (single core, about an hour)

The two configurations of the paper's MVP tables that the oracle can still
finish on one core (§6.1.1 and §6.2.1; points uniform in C = [-1, 1]^d, the
domain of the paper's experiments, passed to the tree explicitly):

* 2D log r, n_max = 100, N = 102400 (kappa 5), eps = 1e-8 -- the paper prints
  RE_MVP = 1.82e-8 for H2*(b+t);
* 3D 1/r, n_max = 125, N = 64000 (kappa 3), eps = 1e-6 -- the paper prints
  1.69e-6.

For each it builds the oracle's H2*(b+t), applies it to two N(0, 1) vectors
and records RE_MVP = ||K~ q - K q|| / ||K q|| against the full dense product
(the paper averages five vectors).  Seeds: points 1100 + d, vectors 2100 + d.
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dense, h2  # noqa: E402
from paper_2309_14085_gb300 import inputs  # noqa: E402

CONFIGS = [  # d, kernel, N, n_max, eps, the paper's RE_MVP
    (2, "log2d", 102400, 100, 1e-8, 1.82e-8),
    (3, "invr", 64000, 125, 1e-6, 1.69e-6),
]


def run(d, kind, N, n_max, eps):
    P = inputs.points(N, d, 1100 + d)
    Q = inputs.rhs(N, 2, 2100 + d)
    t0 = time.time()
    H = h2.H2(P, kind, n_max=n_max, eps=eps, domain=(np.full(d, -1.0), 2.0))
    t1 = time.time()
    Y = H.matvec(Q)
    X = dense.product(kind, P, Q)
    res = [dense.relative_error(Y[:, c], X[:, c]) for c in range(Q.shape[1])]
    return float(np.mean(res)), t1 - t0, H.tree.kappa


def main():
    only = sys.argv[1:]
    out = os.path.join(HERE, "oracle_re_paper_configs.txt")
    lines = []
    for (d, kind, N, n_max, eps, paper) in CONFIGS:
        if only and str(d) not in only:
            continue
        re, tb, kappa = run(d, kind, N, n_max, eps)
        lines.append("%d %s %d %d %.0e %d %.6e %.3e %.0f\n" % (d, kind, N, n_max, eps, kappa, re,
                                                               paper, tb))
        print(lines[-1], end="", flush=True)
    with open(out, "w") as f:
        f.write("# RE_MVP of the oracle's H2*(b+t) at the paper's MVP configurations (written by\n")
        f.write("# tests/golden/make_paper_configs.py from the oracle only; mean of two N(0,1) q,\n")
        f.write("# domain [-1,1]^d).  The paper's value is from the tables of §6.1.1 / §6.2.1.\n")
        f.write("# columns: d kernel N n_max eps kappa oracle_RE paper_RE build_seconds\n")
        f.writelines(lines)
    print(out)


if __name__ == "__main__":
    main()
