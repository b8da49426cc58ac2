"""The plain definition phi = K q (the paper's direct MVP, t_direct in the notation table of §6).

``product`` forms the full product row block by row block; ``rows`` evaluates
selected exact rows only (what large-N checks sample).  RE_MVP is the 2-norm
relative error of the notation table of §6.
"""

import numpy as np

from . import kernels


def rows(kind, P, Q, row_idx, param=0.1, chunk=256):
    """Exact rows (K Q)[row_idx, :] for Q of shape (N,) or (N, nrhs)."""
    Q2 = Q.reshape(Q.shape[0], -1)
    row_idx = np.asarray(row_idx, dtype=np.int64)
    out = np.zeros((row_idx.size, Q2.shape[1]))
    cols = np.arange(P.shape[0])
    for s in range(0, row_idx.size, chunk):
        r = row_idx[s:s + chunk]
        out[s:s + chunk] = kernels.block(kind, P, r, cols, param) @ Q2
    return out.reshape((row_idx.size,) + Q.shape[1:])


def product(kind, P, Q, param=0.1, chunk=256):
    """Full dense product K Q."""
    return rows(kind, P, Q, np.arange(P.shape[0]), param, chunk)


def matrix(kind, P, param=0.1):
    n = P.shape[0]
    return kernels.block(kind, P, np.arange(n), np.arange(n), param)


def relative_error(approx, exact):
    """RE_MVP = ||approx - exact||_2 / ||exact||_2 (notation table of §6)."""
    return float(np.linalg.norm(approx - exact) / np.linalg.norm(exact))
