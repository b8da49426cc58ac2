"""Batched products over many independent trees (one captured CUDA graph of
merged level-synchronous launches) against each matrix applied on its own."""

import numpy as np
import pytest

from oracle import dense, h2
from paper_2309_14085_gb300 import H2Batch, H2Matrix, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["f32", "f64", "df64"])
def test_batch_equals_individual_products(storage):
    rng = np.random.default_rng(3000)
    specs = [(2, 1200, 1), (3, 5000, 2), (2, 9000, 7), (3, 900, 1), (2, 20000, 5), (3, 12000, 3)]
    mats, xs, nr = [], [], []
    for k, (d, N, r) in enumerate(specs):
        P = inputs.points(N, d, 3000 + k, lo=0.0, hi=1.0)
        mats.append(H2Matrix(P, "log2d" if d == 2 else "invr", leaf_size=64, tol=1e-8,
                             storage=storage, near="stored"))
        xs.append(torch.tensor(inputs.rhs(N, r, 4000 + k).reshape(N, r), device="cuda:0"))
        nr.append(r)
    B = H2Batch(mats, nr)
    info = B.info()
    nt = 4 if storage == "f32" else 2                # RHS columns per virtual instance
    assert info["instances"] == 6 and info["virtual_instances"] == sum(-(-r // nt) for r in nr)
    assert info["points_times_rhs"] == sum(s[1] * s[2] for s in specs)
    kmax = max(m.info()["kappa"] for m in mats)
    assert info["launches_per_product"] <= 2 * kmax + 4
    for rep in range(2):                      # the graph replays with fresh inputs
        ys = B.matvec(xs)
        torch.cuda.synchronize()
        for m, x, y in zip(mats, xs, ys):
            ref = m.matvec(x).reshape(y.shape)
            a, b = y.cpu().numpy(), ref.cpu().numpy()
            tol = 1e-6 if storage == "f32" else 1e-12
            assert np.abs(a - b).max() <= tol * np.abs(b).max()
        xs = [x * 0.5 + 1.0 for x in xs]
    # one instance against the oracle
    P = inputs.points(5000, 3, 3001, lo=0.0, hi=1.0)
    q = inputs.rhs(5000, 2, 4001).reshape(5000, 2)
    ref = h2.H2(P, "invr", n_max=64, eps=1e-8).matvec(q)
    got = B.matvec([torch.tensor(inputs.rhs(s[1], s[2], 4000 + k).reshape(s[1], s[2]), device="cuda:0")
                    for k, s in enumerate(specs)])[1].cpu().numpy()
    if storage == "f64":
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    else:
        # every stored entry rounded to a 24 / 48-bit significand: 64 u (|K||q|)_i
        u = 2.0 ** -24 if storage == "f32" else 2.0 ** -48
        absKq = np.abs(dense.matrix("invr", P)) @ np.abs(q)
        assert np.all(np.abs(got - ref) <= 64 * u * absKq)


def test_batch_from_host_only_and_released_handles():
    """A batch takes each instance's operators from the device copy when the
    handle is on the device (its host copy may be released) and from the host
    copy of a host-only handle; both give the instance's own product."""
    specs = [(2, 3000, 1), (3, 4000, 2)]
    pts = [inputs.points(N, d, 3100 + k, lo=0.0, hi=1.0) for k, (d, N, r) in enumerate(specs)]
    kinds = ["log2d", "invr"]
    host = H2Matrix(pts[0], kinds[0], leaf_size=64, tol=1e-8, storage="f32", near="stored",
                    host_only=True)
    dev = H2Matrix(pts[1], kinds[1], leaf_size=64, tol=1e-8, storage="f32", near="stored")
    dev.release_host()
    with pytest.raises(Exception):
        dev.convert("f64")                     # the host operators are gone
    B = H2Batch([host, dev], [1, 2])
    xs = [torch.tensor(inputs.rhs(N, r, 4100 + k).reshape(N, r), device="cuda:0")
          for k, (d, N, r) in enumerate(specs)]
    ys = B.matvec(xs)
    torch.cuda.synchronize()
    for k, (d, N, r) in enumerate(specs):
        ref_m = H2Matrix(pts[k], kinds[k], leaf_size=64, tol=1e-8, storage="f32", near="stored")
        ref = ref_m.matvec(xs[k]).reshape(ys[k].shape).cpu().numpy()
        got = ys[k].cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()


def test_tensor_core_batch_streams_each_instance_once_and_matches_the_oracle():
    """fp32 handles built with tensor cores: the batch runs every step of every
    instance on the tensor cores in 16-column tiles, one virtual instance per
    instance (its operators stream once for all of its 1-16 columns; columns
    past an instance's own are never read).  Every instance is checked against
    the oracle's construction and MVP under the bar of the 3-term tf32 product,
    64 u (|K||q|)_i with u = 2^-20, and the graph replays with new inputs.  The
    bar models zero-mean right-hand sides, as every parity bar here does: with
    a common offset the rounding of the interpolation operators (entries that
    cancel, condition ~1/eps) adds up coherently along the nested chain and
    exceeds it (by 9-27x measured), in the fp32 products as well."""
    rng = np.random.default_rng(3300)
    specs = [(2, 1500, 1), (3, 2600, 7), (2, 5000, 16), (3, 900, 3), (2, 7000, 12), (3, 4000, 2)]
    pts, mats, xs = [], [], []
    for k, (d, N, r) in enumerate(specs):
        P = inputs.points(N, d, 3300 + k, lo=0.0, hi=1.0)
        pts.append(P)
        mats.append(H2Matrix(P, "log2d" if d == 2 else "invr", leaf_size=64, tol=1e-8, storage="f32",
                             near="stored", tensor_cores=True))
        xs.append(torch.tensor(inputs.rhs(N, r, 4300 + k).reshape(N, r), device="cuda:0"))
    B = H2Batch(mats, [s[2] for s in specs])
    info = B.info()
    assert info["instances"] == len(specs) and info["virtual_instances"] == len(specs)
    for rep in range(2):
        ys = B.matvec(xs)
        torch.cuda.synchronize()
        for k, (d, N, r) in enumerate(specs):
            kind = "log2d" if d == 2 else "invr"
            q = xs[k].cpu().numpy()
            ref = h2.H2(pts[k], kind, n_max=64, eps=1e-8).matvec(q).reshape(N, r)
            got = ys[k].cpu().numpy().reshape(N, r)
            bar = 64 * 2.0 ** -20 * (np.abs(dense.matrix(kind, pts[k])) @ np.abs(q)).reshape(N, r)
            ratio = float((np.abs(got - ref) / bar).max())
            print(f"batch tc instance {k} (d {d}, N {N}, {r} RHS): {ratio:.3f} of the bar")
            assert ratio <= 1.0
        xs = [torch.tensor(inputs.rhs(N, r, 4400 + k).reshape(N, r), device="cuda:0")
              for k, (d, N, r) in enumerate(specs)]
