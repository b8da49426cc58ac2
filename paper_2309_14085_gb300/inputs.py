"""Seeded synthetic inputs shaped like the paper's experiments.

This module holds random-number generation only, none of the method's
arithmetic; the tests and the benchmark hand its arrays both to the CUDA
library and to the FP64 oracle.

The paper's MVP experiments draw N points i.i.d. uniform in [-1, 1]^d (§6.1.1
for 2D, §6.2.1 for 3D) and random charge vectors q (averaged over 5 draws).
Here: NumPy PCG64 streams; points U[lo, hi]^d, right-hand sides N(0, 1).
Seeds: points 1000 + workload number, right-hand sides 2000 + workload number,
instance k of the batched workload 3000 + k.
"""

import numpy as np

#: Named workloads (sizes, kernel, tolerance) of the benchmarked configurations.
WORKLOADS = {
    # 2D log r, N = 4096, quadtree with leaves of <= 64 points on average (kappa 3)
    "c1_2d_log_n4096": dict(number=1, N=4096, d=2, kernel="log2d", n_max=64, eps=1e-8, nrhs=1),
    # 3D 1/r, N = 262144, octree kappa 4
    "c2_3d_invr_n262144": dict(number=2, N=262144, d=3, kernel="invr", n_max=64, eps=1e-6, nrhs=1),
    "c2_3d_invr_n262144_eps1e-9": dict(number=2, N=262144, d=3, kernel="invr", n_max=64,
                                        eps=1e-9, nrhs=1),
    # the same kernel and leaf size one level shallower (kappa 3): the profiling case
    "c2s_3d_invr_n32768": dict(number=2, N=32768, d=3, kernel="invr", n_max=64, eps=1e-6, nrhs=1),
    # 2D log r, N = 2^20, kappa 7, 64 right-hand sides
    "c3_2d_log_n1048576": dict(number=3, N=1 << 20, d=2, kernel="log2d", n_max=64, eps=1e-10,
                                nrhs=64),
    # the same kernel, tolerance and RHS count at N = 2^16 (kappa 5): the profiling case
    "c3s_2d_log_n65536": dict(number=3, N=1 << 16, d=2, kernel="log2d", n_max=64, eps=1e-10,
                               nrhs=64),
}


def points(N, d, seed, lo=-1.0, hi=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=(N, d))


def rhs(N, nrhs, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    q = rng.standard_normal(size=(nrhs, N)).T.copy()   # column-major N x nrhs
    return q[:, 0].copy() if nrhs == 1 else q


def workload(name):
    w = dict(WORKLOADS[name])
    w["points"] = points(w["N"], w["d"], 1000 + w["number"])
    w["q"] = rhs(w["N"], w["nrhs"], 2000 + w["number"])
    return w


def batched_instances(count=512, seed0=3000):
    """The batched workload: instance k has N = floor(exp(U[ln 1024, ln 65536]))
    points uniform in the unit square (k even, log r) or cube (k odd, 1/r),
    1 + (k mod 16) right-hand sides N(0, 1); all streams seeded with 3000 + k."""
    out = []
    for k in range(count):
        rng = np.random.Generator(np.random.PCG64(seed0 + k))
        N = int(np.floor(np.exp(rng.uniform(np.log(1024), np.log(65536)))))
        d = 2 if k % 2 == 0 else 3
        P = rng.uniform(0.0, 1.0, size=(N, d))
        r = 1 + (k % 16)
        q = rng.standard_normal(size=(r, N)).T.copy()
        out.append(dict(k=k, N=N, d=d, kernel="log2d" if d == 2 else "invr", points=P, q=q,
                        nrhs=r))
    return out



def served_geometries(count=4, seed0=4000, n_max_3d=32768):
    """Geometries of the served-solves workload: geometry k has points uniform
    in [-1, 1]^d (d = 2 for even k, 3 for odd k) with N = floor(exp(U[ln 4096,
    ln N_hi])), N_hi = 2^20 in 2D and n_max_3d in 3D, and the right-hand side
    f(x) = sin(3 x_1) cos(2 x_2) at the points; streams seeded with 4000 + k."""
    out = []
    for k in range(count):
        rng = np.random.Generator(np.random.PCG64(seed0 + k))
        d = 2 if k % 2 == 0 else 3
        hi = 2 ** 20 if d == 2 else n_max_3d
        N = int(np.floor(np.exp(rng.uniform(np.log(4096), np.log(hi)))))
        P = rng.uniform(-1.0, 1.0, size=(N, d))
        f = np.sin(3.0 * P[:, 0]) * np.cos(2.0 * P[:, 1])
        out.append(dict(k=k, N=N, d=d, points=P, f=f))
    return out


def poisson_arrivals(count, rate, ngeom, seed=4999):
    """Request stream: arrival times (s) of a Poisson process of the given rate
    and the geometry each request targets (uniform)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    g = rng.integers(0, ngeom, size=count)
    return t - t[0], g


def uniform_grid(n, d):
    """Collocation points of the integral-equation experiments: the centres
    -1 + (2 i + 1) / n, i < n, of the n^d cells of a uniform grid on [-1, 1]^d
    (cell measure (2 / n)^d), in lexicographic order."""
    x = -1.0 + (2.0 * np.arange(n) + 1.0) / n
    g = np.meshgrid(*([x] * d), indexing="ij")
    return np.stack([a.ravel() for a in g], axis=1)


def chebyshev_grid(n, d):
    """The n^d tensor grid of Chebyshev points cos(pi (2i + 1) / (2n)), i < n, in
    [-1, 1]^d: the non-uniform point sets of the paper's Chebyshev experiments
    (dense near the faces, sparse in the middle), in lexicographic order."""
    x = np.cos(np.pi * (2 * np.arange(n) + 1) / (2 * n))
    g = np.meshgrid(*([x] * d), indexing="ij")
    return np.stack([a.ravel() for a in g], axis=1)
