"""M2L coupling blocks formed on the device (m2l_mode 2).

T_{X,Y} = G(t^{X,i}, t^{Y,i}) (§3.6.4) is a kernel block between pivot
points, so the device can write the stored blocks from the pivot coordinates
instead of receiving them from the host.  The fill kernel takes the host's
operations in the host's order with every fp64 operation rounded on its own
(squares summed in coordinate order, then sqrt and divisions, all IEEE
correctly rounded), so for 1/r and the IMQ its entries equal the host's bit
for bit and so do the products (the (H2+H)* low-rank sums use atomics, so
there only to rounding); log r and exp(-r) go through the device's libm,
within an ulp of the host's, so there the products agree to rounding.
The host-formed path is the one tested against the oracle elsewhere; equality
with it carries that parity over.
"""

import pytest

from paper_2309_14085_gb300 import H2Batch, H2Matrix, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pair(P, kind, **kw):
    S = H2Matrix(P, kind, leaf_size=64, tol=1e-8, **kw)
    D = H2Matrix(P, kind, leaf_size=64, tol=1e-8, m2l="device", **kw)
    return S, D


# (kind, d, N, variant, storage, nrhs, near, bit-equal or relative bar)
CASES = [
    ("invr", 3, 6000, "h2star", "f64", 1, None, 0.0),
    ("imq", 2, 6000, "h2sqrt", "df64", 1, "stored", 0.0),
    ("invr", 3, 6000, "h2plush", "f32", 3, None, 1e-5),           # low-rank sums: atomics
    ("imq", 3, 6000, "h2star", "bf16", 16, "stored", 0.0),       # 16 RHS: tensor cores
    ("log2d", 2, 6000, "h2star", "f64", 1, None, 1e-12),
    ("matern12", 3, 6000, "h2star_t", "f64", 2, None, 1e-12),
    ("log2d", 2, 6000, "h2sqrt_t", "f32", 1, None, 1e-5),
]


@pytest.mark.parametrize("kind,d,N,variant,storage,nrhs,near,bar", CASES)
def test_device_formed_m2l_matches_the_host_formed_product(kind, d, N, variant, storage, nrhs,
                                                           near, bar):
    P = inputs.points(N, d, 71)
    kp = 0.5 if kind == "imq" else None
    S, D = _pair(P, kind, variant=variant, storage=storage, near=near, kparam=kp)
    assert D.info()["m2l_fly"] == 2 and D.info()["bytes_m2l"] == S.info()["bytes_m2l"]
    X = torch.tensor(inputs.rhs(N, nrhs, 72).reshape(N, nrhs), device="cuda:0")
    ys, yd = S.matvec(X), D.matvec(X)
    torch.cuda.synchronize()
    assert torch.isfinite(yd).all()
    rel = float((yd - ys).abs().max() / ys.abs().max())
    print(f"{kind} {variant} {storage}: max |device - host| / max |y| = {rel:.2e}")
    if bar == 0.0:
        assert torch.equal(ys, yd), rel
    else:
        assert rel <= bar, rel


def test_conversion_and_batching_of_a_device_formed_operator():
    P = inputs.points(5000, 3, 73)
    S, D = _pair(P, "invr", near="stored")
    x = torch.tensor(inputs.rhs(5000, 1, 74), device="cuda:0")
    # a converted copy forms its blocks again, in the target storage
    Sf, Df = S.convert("f32"), D.convert("f32")
    assert torch.equal(Sf.matvec(x), Df.matvec(x))
    # batches copy the device operators, M2L region included
    P2 = inputs.points(3000, 3, 75)
    S2, D2 = _pair(P2, "invr", near="stored")
    x2 = torch.tensor(inputs.rhs(3000, 1, 76), device="cuda:0")
    bs, bd = H2Batch([S, S2]), H2Batch([D, D2])
    ys, yd = bs.matvec([x, x2]), bd.matvec([x, x2])
    torch.cuda.synchronize()
    for a, b in zip(ys, yd):
        assert torch.equal(a, b)
