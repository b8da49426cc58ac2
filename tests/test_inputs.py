"""The seeded synthetic inputs (the workloads' recipes): shapes, ranges,
determinism and the documented distributions."""

import numpy as np

from paper_2309_14085_gb300 import inputs


def test_points_and_rhs_are_seeded_uniform_and_normal():
    a, b = inputs.points(5000, 3, 7), inputs.points(5000, 3, 7)
    assert np.array_equal(a, b) and a.shape == (5000, 3)
    assert a.min() >= -1.0 and a.max() <= 1.0 and abs(a.mean()) < 0.05
    q = inputs.rhs(20000, 2, 9).reshape(20000, 2)
    assert abs(q.mean()) < 0.05 and abs(q.std() - 1.0) < 0.05


def test_workloads_match_their_names():
    for name, spec in inputs.WORKLOADS.items():
        assert f"n{spec['N']}" in name and f"{spec['d']}d" in name
    w = inputs.workload("c3_2d_log_n1048576")
    assert w["N"] == 1 << 20 and w["nrhs"] == 64 and w["eps"] == 1e-10


def test_batched_instances_recipe():
    inst = inputs.batched_instances(64)
    assert [i["k"] for i in inst] == list(range(64))
    for i in inst:
        assert 1024 <= i["N"] < 65536
        assert i["d"] == (2 if i["k"] % 2 == 0 else 3)
        assert i["kernel"] == ("log2d" if i["d"] == 2 else "invr")
        assert i["nrhs"] == 1 + i["k"] % 16 and i["q"].shape == (i["N"], i["nrhs"])
        assert i["points"].min() >= 0.0 and i["points"].max() <= 1.0


def test_served_workload_recipe():
    geo = inputs.served_geometries(6)
    for g in geo:
        assert 4096 <= g["N"] <= (2 ** 20 if g["d"] == 2 else 32768)
        x = g["points"]
        assert np.allclose(g["f"], np.sin(3 * x[:, 0]) * np.cos(2 * x[:, 1]))
    t, gid = inputs.poisson_arrivals(4000, 200.0, 6)
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    assert abs(len(t) / t[-1] - 200.0) < 10.0              # mean rate
    assert set(np.unique(gid)) == set(range(6))


def test_chebyshev_grid():
    g = inputs.chebyshev_grid(5, 2)
    x = np.cos(np.pi * (2 * np.arange(5) + 1) / 10)
    assert g.shape == (25, 2)
    assert np.allclose(np.unique(g[:, 0]), np.sort(x))
    assert np.array_equal(g[:5, 0], np.full(5, x[0])) and np.allclose(g[:5, 1], x)


def test_uniform_grid():
    for n, d in [(64, 2), (16, 3)]:
        g = inputs.uniform_grid(n, d)
        assert g.shape == (n ** d, d)
        h = 2.0 / n
        # cell centres: one per cell, half a cell from the faces, spacing h
        assert np.allclose(g.min(0), -1 + h / 2) and np.allclose(g.max(0), 1 - h / 2)
        assert len(np.unique(np.round(g / h, 6), axis=0)) == n ** d
        assert np.allclose(np.diff(np.unique(g[:, 0])), h)
        # with n a power of two no centre lies on a box boundary of any level
        for level in range(1, int(np.log2(n)) + 1):
            t = (g + 1.0) * 2 ** level / 2.0
            assert np.all(np.abs(t - np.round(t)) > 1e-9)
