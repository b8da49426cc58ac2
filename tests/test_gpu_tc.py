"""Tensor-core products (tcgen05): bfloat16 storage and fp32 storage on the
tensor cores, through the C ABI.

Bars follow the fp32 parity bar of test_gpu_parity.py, |y_i - ref_i| <=
64 u (|K||q|)_i, with u the relative rounding of one product in the format
that limits it: u = 2^-8 for bfloat16 operators (8-bit significand) and
u = 2^-20 for fp32 operators on the 3-term tf32 product (a = a_hi + a_lo,
b = b_hi + b_lo with tf32 hi terms; the dropped a_lo b_lo and the tf32
rounding of the lo terms leave ~2^-21 per product).  The reference is the
oracle's own construction and MVP in fp64 (same pivots, so the difference is
rounding only).  A bf16 tensor-core product rounds the coefficients of every
stage to bf16 as well as the operators, so its bar against the oracle is 2 x
and it is also compared with the CUDA-core product of the same handle.

bf16 operators leave the 2D log r products of these tolerances without a
correct digit (the nested pivot bases carry entries that cancel, with
condition ~1/eps, and log r sums cancel ~20x): bf16 is an inner operator for
iterative refinement there (test_bf16_refinement_reaches_the_fp64_tolerance),
and its relative-error bar applies to 3D 1/r only.
"""

import numpy as np
import pytest

from oracle import dense, h2, kernels
from paper_2309_14085_gb300 import H2Matrix, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda:0")


def _ratio(y, ref, bound):
    return float((np.abs(y - ref) / bound).max())


def _case(kind, d, N, nrhs, seed):
    P = inputs.points(N, d, seed)
    Q = inputs.rhs(N, nrhs, seed + 1).reshape(N, nrhs)
    ref = h2.H2(P, kind, n_max=64, eps=1e-8).matvec(Q)
    absKq = np.abs(dense.matrix(kind, P)) @ np.abs(Q)
    return P, Q, ref.reshape(N, nrhs), absKq


@pytest.mark.parametrize("kind,d", [("log2d", 2), ("invr", 3)])
def test_bf16_storage_matches_the_oracle(kind, d):
    N = 6000
    P, Q, ref, absKq = _case(kind, d, N, 64, 31)
    A = H2Matrix(P, kind, leaf_size=64, tol=1e-8, storage="bf16")
    bar = 64 * 2.0 ** -8 * absKq
    Y = A.matvec(_dev(Q)).cpu().numpy()                      # 64 RHS: tensor cores
    y1 = np.stack([A.matvec(_dev(Q[:, c])).cpu().numpy() for c in range(3)], 1)   # CUDA cores
    r_tc, r_cc = _ratio(Y, ref, 2 * bar), _ratio(y1, ref[:, :3], bar[:, :3])
    r_x = _ratio(Y[:, :3], y1, 2 * bar[:, :3])
    re = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
    print(f"bf16 {kind}: tc {r_tc:.3f}, cuda cores {r_cc:.3f}, tc vs cc {r_x:.3f} of the bar; "
          f"RE vs oracle {re:.2e}")
    assert np.all(np.isfinite(Y))
    assert r_tc <= 1.0 and r_cc <= 1.0 and r_x <= 1.0
    if kind == "invr":
        assert re <= 1e-2


@pytest.mark.parametrize("nrhs", [64, 40, 16, 21])
def test_fp32_tensor_cores_match_the_oracle(nrhs):
    """3-term tf32 tiles of 64 / 32 / 16 columns plus CUDA-core remainders."""
    N = 5000
    P, Q, ref, absKq = _case("log2d", 2, N, nrhs, 41)
    A = H2Matrix(P, "log2d", leaf_size=64, tol=1e-8, storage="f32", near="stored",
                 tensor_cores=True)
    Y = A.matvec(_dev(Q)).cpu().numpy().reshape(N, nrhs)
    r = _ratio(Y, ref, 64 * 2.0 ** -20 * absKq)
    re = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
    print(f"tf32x3 nrhs {nrhs}: {r:.3f} of the bar; RE vs oracle {re:.2e}")
    assert r <= 1.0
    assert re <= 1e-4
    # columns beyond the tensor-core tiles run on the CUDA cores in fp32
    tc_cols = 64 * (nrhs // 64) + 32 * ((nrhs % 64) // 32) + 16 * ((nrhs % 32) // 16)
    if tc_cols < nrhs:
        B = H2Matrix(P, "log2d", leaf_size=64, tol=1e-8, storage="f32", near="stored")
        Z = B.matvec(_dev(Q)).cpu().numpy().reshape(N, nrhs)
        assert np.array_equal(Y[:, tc_cols:], Z[:, tc_cols:])


def test_bf16_refinement_reaches_the_fp64_tolerance():
    P = inputs.points(20000, 2, 51)
    A = H2Matrix(P, "log2d", leaf_size=64, tol=1e-8)
    L = A.convert("bf16")
    b = torch.tensor(inputs.rhs(20000, 1, 52), device="cuda:0")
    x, st = L.gmres(b, shift=1.0, scale=1.0 / 20000, rtol=1e-8, restart=50, maxit=500, residual=A)
    print("bf16 refined:", st)
    assert st["converged"] == 1 and st["fallback"] == 0 and st["rel_residual"] <= 1e-8
    r = b - (x + A.matvec(x) / 20000)
    assert float(torch.linalg.norm(r) / torch.linalg.norm(b)) <= 1.01e-8


def test_bf16_c3_sampled_rows_against_the_exact_product():
    """The 64-RHS workload: 2D log r, N = 2^20, eps 1e-10, bf16 operators; 8
    sampled rows x 64 RHS against the exact product (the oracle's dense rows).
    Reported error; bound: the bf16 bar on each sampled entry."""
    w = inputs.workload("c3_2d_log_n1048576")
    P, Q = w["points"], w["q"].reshape(w["N"], 64)
    A = H2Matrix(P, "log2d", leaf_size=64, tol=1e-10, storage="bf16")
    Y = A.matvec(_dev(Q)).cpu().numpy()
    idx = np.random.default_rng(7).choice(w["N"], 8, replace=False)
    exact = dense.rows("log2d", P, Q, idx)
    absrow = np.abs(kernels.block("log2d", P, idx, np.arange(w["N"]))) @ np.abs(Q)
    r = _ratio(Y[idx], exact, 2 * 64 * 2.0 ** -8 * absrow)
    re = np.linalg.norm(Y[idx] - exact) / np.linalg.norm(exact)
    print(f"c3 bf16: {r:.3f} of the bar; RE on sampled rows {re:.2e}")
    assert r <= 1.0


def test_fp32_tensor_cores_c3_sampled_rows_against_the_exact_product():
    """The 64-RHS workload (2D log r, N = 2^20, eps 1e-10) with fp32 operators on
    the tensor cores (3-term tf32): 8 sampled rows x 64 RHS against the exact
    product (the oracle's dense rows), under the bar of the 3-term product.
    Storing the operators of eps = 1e-10 in fp32 (pivot matrices with condition
    ~1/eps) limits any fp32 product to a few 1e-4 here; the relative error must
    stay below 1e-3."""
    w = inputs.workload("c3_2d_log_n1048576")
    P, Q = w["points"], w["q"].reshape(w["N"], 64)
    A = H2Matrix(P, "log2d", leaf_size=64, tol=1e-10, storage="f32", near="stored",
                 tensor_cores=True)
    Y = A.matvec(_dev(Q)).cpu().numpy()
    idx = np.random.default_rng(7).choice(w["N"], 8, replace=False)
    exact = dense.rows("log2d", P, Q, idx)
    absrow = np.abs(kernels.block("log2d", P, idx, np.arange(w["N"]))) @ np.abs(Q)
    r = _ratio(Y[idx], exact, 64 * 2.0 ** -20 * absrow)
    re = np.linalg.norm(Y[idx] - exact) / np.linalg.norm(exact)
    print(f"c3 tf32x3: {r:.3f} of the bar; RE on sampled rows {re:.2e}")
    assert r <= 1.0 and re <= 1e-3
