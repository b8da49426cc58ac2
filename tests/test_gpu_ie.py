"""Second-kind Fredholm integral equations solved with GMRES on the device (§6,
the 2D and 3D integral-equation experiments).

sigma(x) + int_C F(x, y) sigma(y) dy = f(x) on C = [-1, 1]^d, with F the
Laplace Green's function, -(1/2pi) log r in 2D and 1/(4pi r) in 3D, is
discretised by piecewise-constant collocation at the cell centres of a uniform
grid: (I + s K) sigma = f with K the kernel matrix of log r (2D) or 1/r (3D),
s = -h^2 / (2pi) or h^3 / (4pi) and h = 2 / n the cell width.  The self-cell
integral of the singular kernel is not given; the diagonal of K is 0 here.

As in the paper's RE_sol, q is random, b = K q is the exact product (dense, up
to rounding), and GMRES (unrestarted) on the compressed operator solves for
lambda; every variant is solved.  Bar: lambda - q = (I + s K~)^{-1} s (K - K~) q
up to the GMRES stopping error, with ||(I + s K~)^{-1}|| close to 1 because
||s K q|| / ||q|| is small (checked below), so ||lambda - q|| / ||q|| stays
below eps + 10 eps_GMRES.
"""

import numpy as np
import pytest

from oracle import dense
from paper_2309_14085_gb300 import H2Matrix, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VARIANTS = ["h2star", "h2plush", "h2sqrt", "h2star_t", "h2sqrt_t"]


@pytest.mark.parametrize("kind,d,n,eps,rtol", [("log2d", 2, 64, 1e-10, 1e-12),
                                              ("invr", 3, 16, 1e-6, 1e-10)])
def test_integral_equation_solution_error(kind, d, n, eps, rtol):
    P = inputs.uniform_grid(n, d)
    N = len(P)
    h = 2.0 / n
    s = -h ** 2 / (2 * np.pi) if d == 2 else h ** 3 / (4 * np.pi)
    q = inputs.rhs(N, 1, 811)
    b = q + s * (dense.matrix(kind, P) @ q)
    assert np.linalg.norm(b - q) / np.linalg.norm(q) < 0.1        # ||s K q|| small
    bd = torch.tensor(b, device="cuda:0")
    for variant in VARIANTS:
        A = H2Matrix(P, kind, leaf_size=64, tol=eps, variant=variant)
        lam, st = A.gmres(bd, shift=1.0, scale=s, rtol=rtol, restart=300, maxit=300)
        re = float(np.linalg.norm(lam.cpu().numpy() - q) / np.linalg.norm(q))
        print(f"{kind} N={N} {variant}: {st['iterations']} iterations, "
              f"{1e3 * st['seconds']:.1f} ms, RE_sol {re:.2e}")
        assert st["converged"] == 1 and st["rel_residual"] < rtol, st
        assert re <= eps + 10 * rtol, (variant, re)
