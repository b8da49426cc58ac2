"""Kernel functions K(x, y) = G(|x - y|) of the paper's experiments (fp64).

* ``log2d``    -- single-layer Laplace in 2D, G(r) = log r (§6.1.1).
* ``invr``     -- single-layer Laplace in 3D, G(r) = 1/r (§6.2.1).
* ``matern12`` -- Matérn covariance with nu = 1/2, G(r) = exp(-r) (App. D).
* ``imq``      -- inverse multiquadric G(r) = 1/sqrt(1 + (r/c)^2); not in the
                  paper, it is the kernel of the served RBF-interpolation solves.

Diagonal: the paper sets K(i, i) = 0 for log r and 1/r (§6.1.1, §6.2.1).  For
exp(-r) and the IMQ the natural value G(0) = 1 is used.  Distinct indices whose
points coincide (r = 0) take the same diagonal value (reading: the paper is
silent about coincident points).

r is formed as sqrt(dx^2 + dy^2 [+ dz^2]) with the squares summed in
coordinate order.
"""

import numpy as np

KINDS = ("log2d", "invr", "imq", "matern12")


def diagonal_value(kind):
    return 0.0 if kind in ("log2d", "invr") else 1.0


def G(kind, r, param=0.1):
    """The radial function G(r) for r > 0."""
    if kind == "log2d":
        return np.log(r)
    if kind == "invr":
        return 1.0 / r
    if kind == "imq":
        return 1.0 / np.sqrt(1.0 + (r / param) ** 2)
    if kind == "matern12":
        return np.exp(-r)
    raise ValueError(f"unknown kernel {kind!r}")


def distances(P, rows, cols):
    """Euclidean distance matrix between points P[rows] and P[cols]."""
    X = P[np.asarray(rows, dtype=np.int64)]
    Y = P[np.asarray(cols, dtype=np.int64)]
    r2 = np.zeros((X.shape[0], Y.shape[0]))
    for k in range(P.shape[1]):
        dk = X[:, k][:, None] - Y[:, k][None, :]
        r2 = r2 + dk * dk
    return np.sqrt(r2)


def block(kind, P, rows, cols, param=0.1):
    """The sub-block K_{rows, cols}; rows/cols are global point indices."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    r = distances(P, rows, cols)
    diag = (r == 0.0) | (rows[:, None] == cols[None, :])
    out = np.empty_like(r)
    ok = ~diag
    out[ok] = G(kind, r[ok], param)
    out[diag] = diagonal_value(kind)
    return out
