"""The allocation-free product h2_matvec_noalloc, called through the C ABI.

Callers that cannot call cudaMalloc while products run (a server that
reserved its device memory budget up front, or code recording a CUDA graph)
use this entry point: its scratch lives in a static device array of the
library.  Here its result must equal the ordinary h2_matvec on the same
handle, within the fp64 parity bar of the other GPU tests, on two calls in a
row (the second call must not see the first call's leftovers), and a handle
whose scratch does not fit the array must be refused with a clear message.
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""

import ctypes

import numpy as np
import pytest

import paper_2309_14085_gb300 as pkg
from paper_2309_14085_gb300 import H2Matrix, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_TOL = 1e-11


def _noalloc():
    L = pkg.lib()
    f = L.h2_matvec_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return L, f


def _call(f, A, x, y):
    s = torch.cuda.current_stream()
    return f(A._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
             ctypes.c_void_p(s.cuda_stream))


@pytest.mark.parametrize("kind,d,N,storage,variant,m2l", [
    ("log2d", 2, 4096, "f64", "h2star", None),
    ("invr", 3, 20000, "df64", "h2star", None),
    ("invr", 3, 20000, "f32", "h2star", None),
    ("log2d", 2, 6000, "f64", "h2plush", None),        # the (H2+H)* scratch after the vectors
    ("invr", 3, 12000, "f32", "h2star", "fly"),        # M2L from the pivot coordinates
    ("log2d", 2, 6000, "f64", "h2star", "device")])    # M2L blocks formed on the device
def test_noalloc_equals_matvec_on_two_calls(kind, d, N, storage, variant, m2l):
    L, f = _noalloc()
    A = H2Matrix(inputs.points(N, d, 500 + d), kind, leaf_size=64, tol=1e-8, storage=storage,
                 variant=variant, m2l=m2l)
    q1 = torch.tensor(inputs.rhs(N, 1, 601), device="cuda:0")
    q2 = torch.tensor(inputs.rhs(N, 1, 602), device="cuda:0")
    for q in (q1, q2):
        ref = A.matvec(q)
        out = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda:0")
        rc = _call(f, A, q, out)
        assert rc == 0, L.h2_last_error().decode()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.abs(a - b).max() <= F64_TOL * np.abs(b).max()


def test_noalloc_refuses_scratch_beyond_its_array():
    L, f = _noalloc()
    N = 1 << 21                      # 2 N coefficients alone exceed 32 MiB in fp64
    A = H2Matrix(inputs.points(N, 2, 700), "log2d", leaf_size=64, tol=1e-2, near="fly")
    x = torch.zeros(N, dtype=torch.float64, device="cuda:0")
    y = torch.zeros(N, dtype=torch.float64, device="cuda:0")
    assert _call(f, A, x, y) == -1
    msg = L.h2_last_error().decode()
    assert "scratch" in msg and str(32 << 20) in msg
    assert _call(f, A, x, y) == -1                     # refused again, no state change
    rc = pkg.lib().h2_matvec(A._h, ctypes.c_void_p(x.data_ptr()), N,
                             ctypes.c_void_p(y.data_ptr()), N, 1,
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0                    # the ordinary entry point still serves it
