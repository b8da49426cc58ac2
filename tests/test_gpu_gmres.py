"""GMRES on the device (fp64 vectors), against the oracle and dense solves.

§6 solves second-kind integral equations and RBF systems with GMRES whose
products use the hierarchical representation.  Here (I + K~/N) x = b (the
second-kind form) and an inverse-multiquadric RBF system (sigma I + K~) c = f.
Bars: the solution of the compressed system vs a dense LU solve of the exact
system within a small multiple of the compression tolerance (the operator
differs from K by ~eps), and the recomputed fp64 relative residual below rtol.
"""

import numpy as np
import pytest

from oracle import dense, gmres, h2
from paper_2309_14085_gb300 import H2Matrix, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda:0")


def test_second_kind_2d_log_matches_dense_solve():
    N = 3000
    P = inputs.points(N, 2, 801)
    b = inputs.rhs(N, 1, 802)
    A = H2Matrix(P, "log2d", leaf_size=32, tol=1e-10)
    x, st = A.gmres(_dev(b), shift=1.0, scale=1.0 / N, rtol=1e-12, restart=50)
    assert st["converged"] == 1 and st["rel_residual"] < 1e-12, st
    xd = gmres.dense_solve(np.eye(N) + dense.matrix("log2d", P) / N, b)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xd) / np.linalg.norm(xd) < 1e-8
    # the oracle's own GMRES with its own compressed operator
    O = h2.H2(P, "log2d", n_max=32, eps=1e-10)
    xo, hist, it = gmres.gmres(lambda v: v + O.matvec(v) / N, b, rtol=1e-12, maxit=100)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) < 1e-10
    assert abs(st["iterations"] - it) <= 2


@pytest.mark.parametrize("storage", ["f32", "df64"])
def test_iterative_refinement_reaches_fp64_tolerance(storage):
    """Inner GMRES on the fast product, residuals in fp64 with an fp64 handle."""
    N = 6000
    P = inputs.points(N, 3, 811)
    b = inputs.rhs(N, 1, 812)
    lo = H2Matrix(P, "invr", leaf_size=32, tol=1e-8, storage=storage)
    hi = H2Matrix(P, "invr", leaf_size=32, tol=1e-8, storage="f64")
    x, st = lo.gmres(_dev(b), shift=1.0, scale=1.0 / N, rtol=1e-10, restart=40, residual=hi)
    assert st["converged"] == 1 and st["rel_residual"] < 1e-10, st
    assert st["refinements"] >= 1 and st["matvecs_residual"] == st["refinements"]
    # the same solution as plain fp64 GMRES on the fp64 handle
    x64, st64 = hi.gmres(_dev(b), shift=1.0, scale=1.0 / N, rtol=1e-10, restart=40)
    a, c = x.cpu().numpy(), x64.cpu().numpy()
    assert np.linalg.norm(a - c) / np.linalg.norm(c) < 1e-8


def test_imq_rbf_system_and_not_converged_path():
    N = 4000
    P = inputs.points(N, 2, 821)
    f = np.sin(3 * P[:, 0]) * np.cos(2 * P[:, 1])
    A = H2Matrix(P, "imq", leaf_size=32, tol=1e-8, kparam=0.1)
    c, st = A.gmres(_dev(f), shift=1e-2, scale=1.0, rtol=1e-8, restart=200, maxit=400)
    assert st["converged"] == 1 and st["rel_residual"] < 1e-8, st
    K = dense.matrix("imq", P, param=0.1)
    # residual with the exact operator: the compressed one differs by ~eps ||K|| ||c||
    cg = c.cpu().numpy()
    res = np.linalg.norm(1e-2 * cg + K @ cg - f) / np.linalg.norm(f)
    bound = 1e-8 + 10 * 1e-8 * np.linalg.norm(K, 2) * np.linalg.norm(cg) / np.linalg.norm(f)
    assert res < bound, (res, bound)
    # two iterations cannot reach 1e-8: not converged, stats still filled
    c2, st2 = A.gmres(_dev(f), shift=1e-2, scale=1.0, rtol=1e-8, restart=200, maxit=2)
    assert st2["converged"] == 0 and st2["iterations"] == 2 and st2["rel_residual"] > 1e-8
