"""Failure detection without a GPU fault.

Every mbarrier wait of the tensor-core products is bounded; on expiry the
kernel records it in the handle's device error flag, frees its TMEM and
returns.  h2_inject_wait_expiry runs that path on demand: one warp waits a
bounded number of rounds on an mbarrier that nothing arrives on.  These tests
check that the expiry reaches the host as H2_E_TIMEOUT through every product
entry point (h2_matvec, h2_gmres, a solve server's requests), that it stays on
the flagged handle, and that the device context keeps working afterwards.
"""

import numpy as np
import pytest

from paper_2309_14085_gb300 import H2Error, H2Matrix, H2Server, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _timeout(call):
    with pytest.raises(H2Error) as e:
        call()
    assert e.value.status == "TIMEOUT", str(e.value)


def test_expired_wait_is_reported_and_the_context_survives():
    N = 8192
    P = inputs.points(N, 2, 61)
    A = H2Matrix(P, "log2d", leaf_size=64, tol=1e-8, storage="bf16")
    other = H2Matrix(P, "log2d", leaf_size=64, tol=1e-8)           # fp64, unflagged
    X = torch.tensor(inputs.rhs(N, 16, 62), device="cuda:0")          # 16 RHS: tensor cores
    Y0 = A.matvec(X)
    y64 = other.matvec(X[:, 0].contiguous())
    torch.cuda.synchronize()
    A.inject_wait_expiry(rounds=1 << 12)
    torch.cuda.synchronize()
    _timeout(lambda: A.matvec(X))
    _timeout(lambda: A.matvec(X[:, 0].contiguous()))
    _timeout(lambda: A.gmres(X[:, 0].contiguous(), shift=1.0, scale=1.0 / N, rtol=1e-4))
    # other handles and new ones keep working on the same context
    y64b = other.matvec(X[:, 0].contiguous())
    B = H2Matrix(P, "log2d", leaf_size=64, tol=1e-8, storage="bf16")
    Y1 = B.matvec(X)
    torch.cuda.synchronize()
    assert torch.equal(y64, y64b)
    rel = float((Y1 - Y0).abs().max() / Y0.abs().max())
    assert np.isfinite(rel) and rel <= 1e-6, rel


def test_injection_needs_a_tensor_core_handle():
    P = inputs.points(4096, 3, 63)
    A = H2Matrix(P, "invr", leaf_size=64, tol=1e-6)                  # fp64: no tensor cores
    with pytest.raises(H2Error) as e:
        A.inject_wait_expiry()
    assert e.value.status == "UNSUPPORTED"
    F = A.convert("f32")                                              # fp32 without tf32
    with pytest.raises(H2Error) as e:
        F.inject_wait_expiry()
    assert e.value.status == "UNSUPPORTED"


def test_server_requests_on_an_expired_operator_stop_with_timeout():
    N = 6000
    P = inputs.points(N, 2, 64)
    A = H2Matrix(P, "imq", leaf_size=64, tol=1e-8, kparam=0.1, storage="bf16")
    A.inject_wait_expiry(rounds=1 << 10)
    torch.cuda.synchronize()
    f = np.sin(3 * P[:, 0]) * np.cos(2 * P[:, 1])
    S = H2Server([A], restart=20, max_active=4)
    t = S.submit(0, f, shift=1.0, scale=1.0 / N, rtol=1e-4, maxit=100)
    _timeout(lambda: S.wait(t))
    _timeout(lambda: S.submit(0, f, shift=1.0, scale=1.0 / N, rtol=1e-4, maxit=100))
    S.close()
    # a healthy operator on the same points still serves
    B = H2Matrix(P, "imq", leaf_size=64, tol=1e-8, kparam=0.1)
    S2 = H2Server([B], restart=50, max_active=4)
    x, st = S2.wait(S2.submit(0, f, shift=1.0, scale=1.0 / N, rtol=1e-8, maxit=500))
    S2.close()
    assert st["converged"] == 1 and st["rel_residual"] <= 1e-8
