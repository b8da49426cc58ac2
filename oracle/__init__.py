"""FP64 CPU oracle for the algebraic H2* fast matrix-vector product.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call,
link or execute this package: only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference leg use it.  It shares no code
with the CUDA path (``paper_2309_14085_gb300``) and imports nothing from it.

What it computes (Khan & Ambikasaran, "New algebraic fast algorithms for
N-body problems in two and three dimensions"):

* ``kernels``  -- the kernel functions of the numerical experiments
                  (§6.1.1 log r, §6.2.1 1/r, App. D Matérn exp(-r)) plus the
                  inverse multiquadric used by the served-solve workload.
* ``dense``    -- the plain definition phi = K q (O(N^2)), full or by rows.
* ``tree``     -- the 2^d uniform tree (§3.1) and the neighbour classes and
                  interaction lists of the §5 notation table (weak admissibility, §3.5) and
                  of the strong admissibility condition with eta = sqrt(d) (§3.3).
* ``aca``      -- partially pivoted ACA with the stopping rule of §3.6.
* ``h2``       -- H2*(b+t) (§5.1: B2T NCA on the far field, Algorithm 1; T2B
                  NCA on vertex-sharing clusters, Algorithm 2; operators §3.6.4;
                  MVP §5.1.2), (H2+H)* (§5.2, Algorithms 3-4) and H2_sqrt(d)(b)
                  (App. A), plus a dense assembly of the compressed matrix.
* ``gmres``    -- unrestarted GMRES (§6, notation-table stopping rule) and a dense
                  LU reference solve.

Everything is plain numpy/scipy in float64.  Library primitives used as
single steps: ``numpy`` matrix-vector products, ``scipy.linalg.lu_factor`` /
``lu_solve`` (LU with partial pivoting) and ``numpy.linalg`` norms.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force, textbook special cases or invariants;
the exact RE_MVP values the paper prints are NOT reproducible (other N,
n_max and random draws), so only their orders of magnitude are checked.
"""

from . import kernels, dense, tree, aca, h2, gmres  # noqa: F401
