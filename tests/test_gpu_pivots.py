"""Pivot search on the device (h2_build_opts.pivots: the default of a device build).

The B2T / T2B pivots are integer decisions (argmax positions and the ACA
stopping rule of §3.6).  The device search takes the host's operations in the
host's order -- kernel values through correctly rounded square roots and
divisions, residual updates in cross order without fused multiply-adds, and
the stopping sums in the host's fixed lane order -- so for 1/r and the IMQ its
pivots must equal the host's index for index, in every variant, and the
products built from them must then be equal bit for bit.  log r and exp(-r)
use the device's log / exp (within an ulp of the host library), so there the
pivots may differ where a comparison is that close (on a Chebyshev grid's
exact ties they do) and the default stays on the host; forced onto the device,
the representation must be as accurate as the host-pivot one.  The host pivots are
themselves pinned to the oracle's index for index (test_abi_cpu.py).
"""

import numpy as np
import pytest

from oracle import dense
from paper_2309_14085_gb300 import H2Matrix, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _all_pivots(A):
    info = A.info()
    out = {}
    for b in range(info["nbases"]):
        for l in range(info["kappa"] + 1):
            for X in range(1 << (info["d"] * l)):
                ti, si = A.pivots(b, l, X)
                if len(ti):
                    out[(b, l, X)] = (ti, si)
    return out


def _matvec(A, q):
    x = torch.from_numpy(q).cuda()
    return A.matvec(x).cpu().numpy()


# (kernel, d, N, n_max, eps, variant): every variant, both exact kernels,
# ragged trees (N not a power of the branching) and a tolerance whose ranks
# pass the first device capacity of 192 crosses
EXACT = [
    ("invr", 3, 6000, 32, 1e-6, "h2star"),
    ("invr", 3, 6000, 32, 1e-6, "h2plush"),
    ("invr", 3, 6000, 32, 1e-6, "h2sqrt"),
    ("invr", 3, 6000, 32, 1e-6, "h2star_t"),
    ("invr", 3, 6000, 32, 1e-6, "h2sqrt_t"),
    ("invr", 3, 6000, 32, 1e-6, "h2star_b"),
    ("imq", 2, 20000, 64, 1e-8, "h2star"),
    ("imq", 3, 9000, 64, 1e-8, "h2star"),
    ("invr", 3, 32768, 64, 1e-10, "h2star"),
]


@pytest.mark.parametrize("kind,d,N,n_max,eps,variant", EXACT)
def test_device_pivots_equal_host_pivots(kind, d, N, n_max, eps, variant):
    P = inputs.points(N, d, 7100 + N)
    H = H2Matrix(P, kind, leaf_size=n_max, tol=eps, variant=variant, pivots="host")
    D = H2Matrix(P, kind, leaf_size=n_max, tol=eps, variant=variant, pivots="device")
    hi, di = H.info(), D.info()
    assert di["pivot_problems_device"] > 0 and hi["pivot_problems_device"] == 0
    ph, pd = _all_pivots(H), _all_pivots(D)
    assert ph.keys() == pd.keys()
    for key in ph:
        assert np.array_equal(ph[key][0], pd[key][0]), key
        assert np.array_equal(ph[key][1], pd[key][1]), key
    q = inputs.rhs(N, 1, 7200 + N).reshape(N)
    assert np.array_equal(_matvec(H, q), _matvec(D, q))
    print(kind, d, N, eps, variant, "problems on the device", di["pivot_problems_device"],
          "on the host", di["pivot_problems_host"], "max rank", max(v[2] for b in di["ranks"] for v in b.values()),
          "pivot seconds host %.2f device %.2f" % (hi["pivot_seconds"], di["pivot_seconds"]))


@pytest.mark.parametrize("kind", ["invr", "imq"])
def test_device_pivots_equal_host_pivots_on_a_chebyshev_grid(kind):
    """18^3 Chebyshev points: a symmetric point set where many residual
    entries tie exactly, so every first-index tie rule is exercised; with
    correctly rounded kernel values the device breaks each tie as the host
    does.  The default of a device build is the device search."""
    P = inputs.chebyshev_grid(18, 3)
    H = H2Matrix(P, kind, leaf_size=32, tol=1e-8, pivots="host")
    D = H2Matrix(P, kind, leaf_size=32, tol=1e-8)
    assert D.info()["pivot_problems_device"] > 0
    ph, pd = _all_pivots(H), _all_pivots(D)
    assert ph.keys() == pd.keys()
    for key in ph:
        assert np.array_equal(ph[key][0], pd[key][0]), key
        assert np.array_equal(ph[key][1], pd[key][1]), key


@pytest.mark.parametrize("kind,d,N,eps", [("log2d", 2, 20000, 1e-8), ("matern12", 3, 9000, 1e-6)])
def test_device_pivots_with_library_log_exp(kind, d, N, eps):
    """log r / exp(-r): pivots agree with the host's up to last-bit kernel
    values, and the representation built from them is as accurate as the
    host-pivot one on 512 rows of the oracle's dense fp64 product."""
    P = inputs.points(N, d, 7300 + N)
    H = H2Matrix(P, kind, leaf_size=64, tol=eps)
    D = H2Matrix(P, kind, leaf_size=64, tol=eps, pivots="device")
    assert H.info()["pivot_problems_device"] == 0     # the default for log r / exp(-r)
    ph, pd = _all_pivots(H), _all_pivots(D)
    same = sum(np.array_equal(ph[k][0], pd.get(k, ([], []))[0]) for k in ph)
    q = inputs.rhs(N, 1, 7400 + N).reshape(N)
    rows = np.random.default_rng(7500).choice(N, 512, replace=False)
    exact = dense.rows(kind, P, q[:, None], rows)[:, 0]
    re_h = np.linalg.norm(_matvec(H, q)[rows] - exact) / np.linalg.norm(exact)
    re_d = np.linalg.norm(_matvec(D, q)[rows] - exact) / np.linalg.norm(exact)
    print(kind, "boxes with equal pivots", same, "of", len(ph), "RE host %.3e device %.3e" % (re_h, re_d))
    assert same >= 0.9 * len(ph)
    assert re_d <= 1.25 * re_h and re_d <= 30 * eps


@pytest.mark.parametrize("kind,d,N,variant", [("invr", 3, 5000, "h2star"), ("invr", 3, 5000, "h2plush"),
                                              ("imq", 2, 6000, "h2plush")])
def test_device_construction_equals_the_hosts_byte_for_byte(tmp_path, kind, d, N, variant):
    """The whole construction written by h2_save -- every pivot, every operator
    and, for (H2+H)*, every kept ACA factor of Algorithm 3 (those pairs run on
    the device too) -- is the same with the device search as with the host's.
    Bytes 60-91 hold the build and pivot-search times and the device / host
    problem counts, the last 8 the checksum."""
    P = inputs.points(N, d, 7700 + N)
    H = H2Matrix(P, kind, leaf_size=32, tol=1e-6, variant=variant, pivots="host")
    D = H2Matrix(P, kind, leaf_size=32, tol=1e-6, variant=variant)
    hi, di = H.info(), D.info()
    assert hi["pivot_problems_device"] == 0
    assert di["pivot_problems_host"] == 0
    assert di["pivot_problems_device"] == hi["pivot_problems_host"]
    if variant == "h2plush":
        assert di["lowrank_pairs"] > 0 and di["bytes_lowrank"] == hi["bytes_lowrank"]
    fa, fb = str(tmp_path / "h.h2"), str(tmp_path / "d.h2")
    H.save(fa)
    D.save(fb)
    a, b = open(fa, "rb").read(), open(fb, "rb").read()
    assert len(a) == len(b) and a[:60] == b[:60] and a[92:-8] == b[92:-8]
