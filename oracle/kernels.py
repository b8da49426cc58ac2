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

log r and exp(-r) come from the platform C library, one call per entry
(``libm.c``, compiled on first use): their last bit depends on the
implementation, and on point sets with exact ties (tensor grids) it decides
the ACA pivots (reading: the paper fixes no implementation; the oracle uses the
C library's, which a C or C++ construction on the same platform shares).
"""

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBM = None
_LIBM_LOCK = threading.Lock()


def _libm():
    """The compiled libm.c (built into oracle/_build/ when missing or stale)."""
    global _LIBM
    with _LIBM_LOCK:
        if _LIBM is None:
            src = os.path.join(_HERE, "libm.c")
            out_dir = os.path.join(_HERE, "_build")
            lib = os.path.join(out_dir, "liboracle_libm.so")
            if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
                os.makedirs(out_dir, exist_ok=True)
                tmp = lib + ".%d.tmp" % os.getpid()
                subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fno-builtin",
                                "-ffp-contract=off", src, "-o", tmp, "-lm"], check=True)
                os.replace(tmp, lib)
            L = ctypes.CDLL(lib)
            for f in (L.oracle_log, L.oracle_exp_neg):
                f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long]
                f.restype = None
            _LIBM = L
    return _LIBM


def _c_elementwise(fn, r):
    r = np.ascontiguousarray(r, dtype=np.float64)
    out = np.empty_like(r)
    fn(r.ctypes.data, out.ctypes.data, r.size)
    return out

KINDS = ("log2d", "invr", "imq", "matern12")


def diagonal_value(kind):
    return 0.0 if kind in ("log2d", "invr") else 1.0


def G(kind, r, param=0.1):
    """The radial function G(r) for r > 0."""
    if kind == "log2d":
        return _c_elementwise(_libm().oracle_log, r)
    if kind == "invr":
        return 1.0 / r
    if kind == "imq":
        return 1.0 / np.sqrt(1.0 + (r / param) ** 2)
    if kind == "matern12":
        return _c_elementwise(_libm().oracle_exp_neg, r)
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
