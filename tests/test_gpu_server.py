"""The continuous-batching solve server: results alone and in the mix,
admission by the workspace budget, and agreement with h2_gmres."""

import threading

import numpy as np
import pytest

from paper_2309_14085_gb300 import H2Matrix, H2Server, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _geoms():
    out = []
    for k, (d, N) in enumerate([(2, 3000), (3, 4000), (2, 6000)]):
        P = inputs.points(N, d, 900 + k)
        out.append((P, H2Matrix(P, "imq", leaf_size=64, tol=1e-8, kparam=0.1)))
    return out


def _rhs(P):
    return np.sin(3 * P[:, 0]) * np.cos(2 * P[:, 1])


def test_results_same_alone_and_in_the_mix():
    G = _geoms()
    mats = [m for _, m in G]
    jobs = [(g, 1e-2 * (1 + k % 3)) for k in range(12) for g in [k % 3]]
    # alone: one request at a time
    alone = {}
    with_server = H2Server(mats, restart=100, max_active=1)
    for k, (g, sigma) in enumerate(jobs):
        t = with_server.submit(g, _rhs(G[g][0]) * (1 + k), shift=sigma, rtol=1e-8, maxit=3000)
        x, st = with_server.wait(t)
        assert st["converged"] == 1 and st["rel_residual"] <= 1e-8, st
        alone[k] = x[:G[g][1].N].copy()
    with_server.close()
    # in the mix: all submitted at once from two threads, up to 8 active
    S = H2Server(mats, restart=100, max_active=8)
    tickets = {}
    def submit(ks):
        for k in ks:
            g, sigma = jobs[k]
            tickets[k] = S.submit(g, _rhs(G[g][0]) * (1 + k), shift=sigma, rtol=1e-8, maxit=3000)
    th = [threading.Thread(target=submit, args=(list(range(i, 12, 2)),)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for k in range(12):
        g = jobs[k][0]
        x, st = S.wait(tickets[k])
        assert st["converged"] == 1 and st["rel_residual"] <= 1e-8, st
        xm = x[:G[g][1].N]
        assert np.abs(xm - alone[k]).max() <= 1e-12 * np.abs(alone[k]).max()
    s = S.stats()
    assert s["completed"] == 12 and s["max_active"] > 1
    assert s["product_columns"] > s["products"]        # products carried several requests
    S.close()


def test_admission_respects_the_workspace_budget_and_matches_gmres():
    G = _geoms()
    mats = [m for _, m in G]
    N = max(m.N for m in mats)
    per = ((100 + 1) + 3) * N * 8 + 304 * 101 * 8 + 101 * 8
    S = H2Server(mats, workspace_bytes=2 * per + 1024, restart=100, max_active=8)
    ts = [S.submit(2, _rhs(G[2][0]), shift=1e-2, rtol=1e-8, maxit=3000) for _ in range(5)]
    xs = [S.wait(t)[0][:mats[2].N] for t in ts]
    s = S.stats()
    assert s["completed"] == 5 and s["max_active"] <= 2
    S.close()
    b = torch.tensor(_rhs(G[2][0]), device="cuda:0")
    x, st = mats[2].gmres(b, shift=1e-2, scale=1.0, rtol=1e-8, restart=100, maxit=3000)
    ref = x.cpu().numpy()
    for xs_ in xs:
        assert np.linalg.norm(xs_ - ref) / np.linalg.norm(ref) <= 1e-5
