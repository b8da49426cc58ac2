"""The continuous-batching solve server: results alone and in the mix,
admission by the workspace budget, agreement with h2_gmres, and
mixed-precision serving (fp32 operators, fp64 residuals) reaching the fp64
tolerance."""

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
    per = ((100 + 1) + 4) * N * 8 + 304 * 101 * 8 + 101 * 8
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


def _true_residual(A, x, f, shift):
    """||f - (shift x + K~ x)|| / ||f|| with the fp64 product, computed here."""
    xt = torch.tensor(x, device="cuda:0")
    r = torch.tensor(f, device="cuda:0") - (shift * xt + A.matvec(xt))
    return float(torch.linalg.norm(r) / np.linalg.norm(f))


def test_mixed_precision_server_reaches_the_fp64_tolerance():
    G = _geoms()
    mats = [m for _, m in G]
    lows = [m.convert("f32") for m in mats]
    jobs = [(k % 3, 1e-2 * (1 + k % 2)) for k in range(6)]
    # one server at a time: a server owns its handles (the fp64 ones serve both)
    plain = H2Server(mats, restart=100, max_active=8)
    tp = [plain.submit(g, _rhs(G[g][0]), shift=s, rtol=1e-8, maxit=6000) for g, s in jobs]
    outp = [plain.wait(t) for t in tp]
    with pytest.raises(Exception):
        H2Server(lows, residual=mats)             # the fp64 handles are taken
    plain.close()
    mixed = H2Server(lows, residual=mats, restart=100, max_active=8)
    tm = [mixed.submit(g, _rhs(G[g][0]), shift=s, rtol=1e-8, maxit=6000) for g, s in jobs]
    outm = [mixed.wait(t) for t in tm]
    mixed.close()
    for (g, s), (xp, sp), (xm, sm) in zip(jobs, outp, outm):
        N = mats[g].N
        xp, xm = xp[:N], xm[:N]
        assert sp["converged"] == 1 and sm["converged"] == 1, (sp, sm)
        assert sm["rel_residual"] <= 1e-8
        assert _true_residual(mats[g], xm, _rhs(G[g][0]), s) <= 1.01e-8
        assert np.linalg.norm(xm - xp) / np.linalg.norm(xp) <= 1e-5
        assert sm["restarts"] >= 1            # at least one fp64 refinement step
        assert sm["op"] in (0, 2)             # fp32 passes the admission rule here


def test_precision_guards_route_requests_to_the_fp64_operator():
    """An inner operator far from the residual operator (IMQ with c = 0.5 against
    c = 0.1, same points) fails the admission rule (op 1); forced onto it, the
    first cycle does not halve the fp64 residual and is undone (op 2); an fp32
    copy passes (op 0).  Every request still reaches the fp64 tolerance."""
    P = inputs.points(3000, 2, 900)
    f = _rhs(P)
    A = H2Matrix(P, "imq", leaf_size=64, tol=1e-8, kparam=0.1)
    W = H2Matrix(P, "imq", leaf_size=64, tol=1e-8, kparam=0.5)
    L = A.convert("f32")
    cases = [(W, 0, 1), (W, 1, 2), (L, 0, 0)]     # (inner, inner_policy, expected op)
    for inner, policy, op in cases:
        S = H2Server([inner], residual=[A], restart=100, max_active=4, inner_policy=policy)
        with pytest.raises(Exception):
            A.matvec(torch.zeros(3000, dtype=torch.float64, device="cuda:0"))  # served handle
        x, st = S.wait(S.submit(0, f, shift=1.0, rtol=1e-8, maxit=3000))
        S.close()
        assert st["converged"] == 1 and st["op"] == op, st
        assert _true_residual(A, x[:3000], f, 1.0) <= 1.01e-8
    # h2_gmres: the same guard finishes the solve with fp64 GMRES
    b = torch.tensor(f, device="cuda:0")
    x, st = W.gmres(b, shift=1.0, rtol=1e-8, restart=100, maxit=3000, residual=A)
    assert st["converged"] == 1 and st["fallback"] == 1, st
    assert _true_residual(A, x.cpu().numpy(), f, 1.0) <= 1.01e-8
    x, st = L.gmres(b, shift=1.0, rtol=1e-8, restart=100, maxit=3000, residual=A)
    assert st["converged"] == 1 and st["fallback"] == 0, st


def test_served_solutions_match_a_dense_solve():
    """Served solutions of (sigma I + K) x = f against a dense LU solve of the
    exact system (the oracle's matrix and solver) on small geometries, for the
    fp64 server and the mixed-precision one (double-float operators, fp64
    residuals).  The bar follows from the perturbation bound
    |x - x*| / |x*| <= cond (|K - K~| / |A| + rtol), with |K - K~| / |A| taken
    as 10 eps and the condition number computed from the dense matrix."""
    from oracle import dense, gmres
    sigma, eps, rtol = 1e-2, 1e-8, 1e-8
    specs = [(2, 1800, 911), (3, 2400, 912)]
    geoms, f64s, dfs = [], [], []
    for d, N, seed in specs:
        P = inputs.points(N, d, seed)
        geoms.append(P)
        A = H2Matrix(P, "imq", leaf_size=48, tol=eps, kparam=0.1)
        f64s.append(A)
        dfs.append(A.convert("df64"))
    for mats, residual in ((f64s, None), (dfs, f64s)):
        S = H2Server(mats, restart=200, max_active=4, residual=residual)
        tickets = [S.submit(g, _rhs(geoms[g]), shift=sigma, rtol=rtol, maxit=5000)
                   for g in range(len(specs))]
        for g, t in enumerate(tickets):
            x, st = S.wait(t)
            assert st["converged"] == 1 and st["rel_residual"] <= rtol, st
            P = geoms[g]
            M = sigma * np.eye(len(P)) + dense.matrix("imq", P, param=0.1)
            xd = gmres.dense_solve(M, _rhs(P))
            cond = np.linalg.cond(M)
            err = np.linalg.norm(x[:len(P)] - xd) / np.linalg.norm(xd)
            bar = cond * (10 * eps + rtol)
            print(f"served {'fp64' if residual is None else 'df64+fp64'} geometry {g}: "
                  f"error vs dense LU {err:.2e}, bar {bar:.2e} (cond {cond:.1e})")
            assert err <= bar
        S.close()
