"""Checkpoints on the device: an operator saved with h2_save and read back with
h2_load gives the products of the saved one bit for bit (the same operators go
through the same kernels), including M2L blocks formed on the device and RHS
tiles on the tensor cores; a handle whose host operators were released cannot
be saved.  A converted copy (which copies the host state the same way) keeps
working after its source is destroyed."""

import pytest

from paper_2309_14085_gb300 import H2Error, H2Matrix, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_loaded_operators_give_the_saved_products(tmp_path):
    N = 6000
    P = inputs.points(N, 3, 95)
    x = torch.tensor(inputs.rhs(N, 1, 96), device="cuda:0")
    X = torch.tensor(inputs.rhs(N, 16, 97).reshape(N, 16), device="cuda:0")
    A = H2Matrix(P, "invr", leaf_size=64, tol=1e-6)
    A.save(str(tmp_path / "a.h2"))
    B = H2Matrix.load(str(tmp_path / "a.h2"))
    assert (B.N, B.d, B.kernel, B.storage) == (N, 3, "invr", "f64")
    assert torch.equal(A.matvec(x), B.matvec(x))
    C = H2Matrix(P, "imq", leaf_size=64, tol=1e-6, storage="bf16", m2l="device", kparam=0.5)
    C.save(str(tmp_path / "c.h2"))
    D = H2Matrix.load(str(tmp_path / "c.h2"))
    assert D.info()["m2l_fly"] == 2
    assert torch.equal(C.matvec(X), D.matvec(X))
    A.release_host()
    with pytest.raises(H2Error) as e:
        A.save(str(tmp_path / "released.h2"))
    assert e.value.status == "UNSUPPORTED"


def test_converted_copy_outlives_its_source():
    """h2_convert copies the host state; the copy's bases refer to its own
    interaction lists, so its statistics stay valid after the source is gone."""
    P = inputs.points(5000, 2, 99)
    S = H2Matrix(P, "log2d", leaf_size=64, tol=1e-8)
    pairs = S.info()["m2l_pairs"]
    F = S.convert("f32")
    S.close()
    assert F.info()["m2l_pairs"] == pairs
    x = torch.tensor(inputs.rhs(5000, 1, 100), device="cuda:0")
    assert torch.isfinite(F.matvec(x)).all()
