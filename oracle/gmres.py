"""GMRES (oracle, fp64) and a dense reference solve.

§6 (notation table): GMRES without restart, stopped when the relative residual
falls below eps_GMRES.  Readings (the paper fixes none of these): x0 = 0;
Arnoldi by modified Gram-Schmidt, re-orthogonalised once when the norm of the
new vector drops below 0.7 of its norm before orthogonalisation; Givens
rotations; the relative residual is ||b - A x||_2 / ||b||_2 as tracked by the
least-squares problem.  RE_sol = ||x - q|| / ||q|| (notation table of §6).
"""

import numpy as np
import scipy.linalg


def gmres(matvec, b, rtol=1e-10, maxit=200):
    """Returns (x, residual history (relative), iterations)."""
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    beta = float(np.linalg.norm(b))
    if beta == 0.0:
        return np.zeros(n), [0.0], 0
    V = np.zeros((maxit + 1, n))
    H = np.zeros((maxit + 1, maxit))
    cs, sn = np.zeros(maxit), np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = beta
    V[0] = b / beta
    hist = [1.0]
    k = 0
    for j in range(maxit):
        w = matvec(V[j])
        norm0 = float(np.linalg.norm(w))
        for i in range(j + 1):
            H[i, j] = float(np.dot(w, V[i]))
            w = w - H[i, j] * V[i]
        if np.linalg.norm(w) < 0.7 * norm0:
            for i in range(j + 1):
                c = float(np.dot(w, V[i]))
                H[i, j] += c
                w = w - c * V[i]
        hnext = float(np.linalg.norm(w))
        H[j + 1, j] = hnext
        for i in range(j):
            h0, h1 = H[i, j], H[i + 1, j]
            H[i, j] = cs[i] * h0 + sn[i] * h1
            H[i + 1, j] = -sn[i] * h0 + cs[i] * h1
        den = np.hypot(H[j, j], H[j + 1, j])
        cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
        H[j, j] = den
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        hist.append(abs(g[j + 1]) / beta)
        if hist[-1] < rtol or hnext == 0.0:
            break
        V[j + 1] = w / hnext
    y = scipy.linalg.solve_triangular(H[:k, :k], g[:k])
    x = V[:k].T @ y
    return x, hist, k


def dense_solve(A, b):
    """Reference solution by LU with partial pivoting."""
    return scipy.linalg.lu_solve(scipy.linalg.lu_factor(A), b)
