"""Pins of the FP64 oracle against things other than itself.

Each test checks an oracle function against a closed form the paper prints,
brute force on tiny inputs, a textbook special case or an invariant of the
mathematics, chosen so that a dropped term, a wrong sign/index or a transposed
operand in the oracle fails at least one of them.
"""

import math
import os

import numpy as np
import pytest

from oracle import aca, dense, gmres, h2, kernels, tree
from paper_2309_14085_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------- kernels
def test_kernel_closed_forms():
    P2 = np.array([[0.0, 0.0], [3.0, 4.0], [0.0, 0.0]])
    K = kernels.block("log2d", P2, [0, 1, 2], [0, 1, 2])
    assert K[0, 1] == pytest.approx(math.log(5.0), rel=1e-15)
    assert K[1, 0] == K[0, 1]
    assert K[0, 0] == 0.0 and K[1, 1] == 0.0      # diagonal 0 (§6.1.1)
    assert K[0, 2] == 0.0                          # coincident points: diagonal value
    P3 = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 2.0]])
    assert kernels.block("invr", P3, [0], [1])[0, 0] == pytest.approx(1.0 / 3.0, rel=1e-15)
    assert kernels.block("invr", P3, [1], [1])[0, 0] == 0.0   # diagonal 0 (§6.2.1)
    assert kernels.block("matern12", P3, [0], [1])[0, 0] == pytest.approx(math.exp(-3.0))
    assert kernels.block("matern12", P3, [0], [0])[0, 0] == 1.0
    Pi = np.array([[0.0, 0.0], [0.1, 0.0]])
    assert kernels.block("imq", Pi, [0], [1], 0.1)[0, 0] == pytest.approx(1 / math.sqrt(2.0))
    assert kernels.block("imq", Pi, [0], [0], 0.1)[0, 0] == 1.0


def test_dense_product_brute_force():
    rng = np.random.default_rng(7)
    for kind, d in [("log2d", 2), ("invr", 3), ("imq", 2), ("matern12", 3)]:
        P = rng.uniform(-1, 1, (23, d))
        q = rng.standard_normal(23)
        phi = dense.product(kind, P, q, chunk=5)
        for i in range(23):
            s = 0.0
            for j in range(23):
                if i == j:
                    kij = kernels.diagonal_value(kind)
                else:
                    r = math.sqrt(sum((P[i, k] - P[j, k]) ** 2 for k in range(d)))
                    kij = {"log2d": math.log(r), "invr": 1 / r,
                           "imq": 1 / math.sqrt(1 + (r / 0.1) ** 2),
                           "matern12": math.exp(-r)}[kind]
                s += kij * q[j]
            assert phi[i] == pytest.approx(s, rel=1e-12, abs=1e-12)
        sub = dense.rows(kind, P, q, [3, 17])
        assert np.allclose(sub, phi[[3, 17]], rtol=1e-14, atol=1e-14)


# --------------------------------------------------------------------------- tree
@pytest.mark.parametrize("N,n_max,d,kappa", [
    (4096, 64, 2, 3), (262144, 64, 3, 4), (1 << 20, 64, 2, 7),
    (102400, 100, 2, 5), (64000, 125, 3, 3), (4097, 64, 2, 4), (10, 64, 2, 0)])
def test_kappa_formula(N, n_max, d, kappa):
    # §3.1: N <= n_max 2^(d kappa) with kappa = ceil(log_{2^d}(N / n_max))
    assert tree.kappa_formula(N, n_max, d) == kappa
    if N > n_max:
        assert kappa == math.ceil(math.log(N / n_max, 2 ** d) - 1e-12)


def test_tree_boxes_contain_points():
    P = inputs.points(3000, 3, 11)
    t = tree.Tree(P, n_max=16)
    h = t.side / (1 << t.kappa)
    lo_box = t.lo + t.leaf_coords * h
    assert np.all(P >= lo_box - 1e-12) and np.all(P <= lo_box + h + 1e-12)
    seen = np.zeros(3000, dtype=int)
    for X in range(t.nboxes(t.kappa)):
        idx = t.points(t.kappa, X)
        seen[idx] += 1
        assert np.all(np.diff(idx[np.argsort(idx)]) > 0)
    assert np.all(seen == 1)
    # a parent's points are its children's, in child order (tree order)
    for X in range(t.nboxes(1)):
        kids = np.concatenate([t.points(2, c) for c in t.children(X)])
        assert np.array_equal(kids, t.points(1, X))


def _max_sizes(d, kappa):
    P = np.zeros((1, d))
    t = tree.Tree(P, n_max=1, kappa=kappa, domain=(np.full(d, -1.0), 2.0))
    m = dict(near=0, far=0, ver=0, star=0, sqrt=0, nsqrt=0)
    for l in range(1, kappa + 1):
        for X in range(t.nboxes(l)):
            f, v = len(t.il_far(l, X)), len(t.il_ver(l, X))
            m["far"] = max(m["far"], f)
            m["ver"] = max(m["ver"], v)
            m["star"] = max(m["star"], f + v)
            m["near"] = max(m["near"], len(t.near_star(l, X)))
            m["sqrt"] = max(m["sqrt"], len(t.il_sqrt(l, X)))
            m["nsqrt"] = max(m["nsqrt"], len(t.near_sqrt(l, X)))
    return m


@pytest.mark.parametrize("row", _golden("list_maxima.txt"))
def test_list_maxima_match_paper(row):
    d, near, star, ver, far, sq, nsq = map(int, row)
    m = _max_sizes(d, 4 if d == 2 else 3)
    assert (m["near"], m["star"], m["ver"], m["far"], m["sqrt"], m["nsqrt"]) == \
        (near, star, ver, far, sq, nsq)
    # the closed forms of §3.5 and Remark 3.1
    assert near == 3 ** d - 2 ** d and star == 6 ** d - 4 ** d - 3 ** d + 2 ** d
    assert ver == 2 ** d - 1 and far == 6 ** d - 4 ** d - 3 ** d + 1
    assert sq == 6 ** d - 3 ** d and nsq == 3 ** d


def _admissible_weak(a, b):
    return tree.classify(a, b) in ("far", "ver")


@pytest.mark.parametrize("d,kappa", [(2, 4), (3, 3)])
def test_lists_are_maximal_admissible_blocks(d, kappa):
    """Independent definition: Y is in IL(X) iff (X, Y) is admissible at level l
    and (parent X, parent Y) is not admissible (or l == 1, where the parents are
    the root).  Also the symmetry Y in IL(X) <=> X in IL(Y)."""
    t = tree.Tree(np.zeros((1, d)), n_max=1, kappa=kappa, domain=(np.full(d, -1.0), 2.0))
    for l in range(1, kappa + 1):
        n = t.nboxes(l)
        coords = [tree.key_to_coords(k, l, d) for k in range(n)]
        step = 1 if n <= 64 else 7          # a sample of targets on the finest 3D level
        for X in range(0, n, step):
            want = set()
            for Y in range(n):
                if not _admissible_weak(coords[X], coords[Y]):
                    continue
                if l > 1:
                    pa = tree.key_to_coords(X >> d, l - 1, d)
                    pb = tree.key_to_coords(Y >> d, l - 1, d)
                    if _admissible_weak(pa, pb):
                        continue
                want.add(Y)
            got = set(t.il_far(l, X)) | set(t.il_ver(l, X))
            assert got == want
            for Y in got:
                assert X in set(t.il_far(l, Y)) | set(t.il_ver(l, Y))


@pytest.mark.parametrize("variant", ["h2star", "h2sqrt"])
def test_block_partition_covers_every_pair_once(variant):
    """Every (target, source) pair lies in exactly one block: a leaf near-field
    block or one admissible pair at exactly one level (brute force, tiny N)."""
    P = inputs.points(300, 2, 5)
    t = tree.Tree(P, n_max=8)
    cover = np.zeros((300, 300), dtype=int)
    for l in range(1, t.kappa + 1):
        for X in range(t.nboxes(l)):
            Ys = (t.il_far(l, X) + t.il_ver(l, X)) if variant == "h2star" else t.il_sqrt(l, X)
            for Y in Ys:
                cover[np.ix_(t.points(l, X), t.points(l, Y))] += 1
    near = t.near_star if variant == "h2star" else t.near_sqrt
    for X in range(t.nboxes(t.kappa)):
        for Y in near(t.kappa, X):
            cover[np.ix_(t.points(t.kappa, X), t.points(t.kappa, Y))] += 1
    assert np.all(cover == 1)


def test_full_grid_pair_counts_2d():
    """Exact counts on a full 8 x 8 quadtree (kappa 3), enumerated directly from
    the box coordinates (vertex-sharing pairs have all |delta| = 1)."""
    t = tree.Tree(np.zeros((1, 2)), n_max=1, kappa=3, domain=(np.full(2, -1.0), 2.0))
    far = {l: sum(len(t.il_far(l, X)) for X in range(t.nboxes(l))) for l in (2, 3)}
    ver = {l: sum(len(t.il_ver(l, X)) for X in range(t.nboxes(l))) for l in (1, 2, 3)}
    # vertex-sharing pairs: at level 1 all 4 diagonal sibling pairs; at level l >= 2 the
    # diagonal pairs whose parents are not themselves diagonal neighbours.
    def diag_pairs(l):
        n = 1 << l
        cnt = 0
        for x in range(n):
            for y in range(n):
                for dx in (-1, 1):
                    for dy in (-1, 1):
                        a, b = x + dx, y + dy
                        if 0 <= a < n and 0 <= b < n:
                            px, py, qx, qy = x >> 1, y >> 1, a >> 1, b >> 1
                            if l == 1 or not (abs(px - qx) == 1 and abs(py - qy) == 1):
                                cnt += 1
        return cnt
    assert ver == {l: diag_pairs(l) for l in (1, 2, 3)}
    assert ver == {1: 4, 2: 32, 3: 160}
    assert far == {2: 96, 3: 576}
    near = sum(len(t.near_star(3, X)) for X in range(t.nboxes(3)))
    assert near == 64 + 2 * (2 * 8 * 7)       # self + both orientations of edge pairs


# --------------------------------------------------------------------------- ACA
def test_aca_exact_low_rank_and_skeleton_form():
    rng = np.random.default_rng(3)
    r = 6
    A = rng.standard_normal((40, r)) @ rng.standard_normal((r, 55))
    rows, cols, U, V = aca.aca_entries(lambda i: A[i], lambda j: A[:, j], 40, 55, 1e-13)
    # r exact crosses; after them every residual row is rounding (below the
    # noise floor), so no further pivot exists
    assert len(rows) == r
    assert np.linalg.norm(A - U @ V.T) <= 1e-12 * np.linalg.norm(A)
    # the cross form of §3.6: U V^* = K_{t,sigma} (K_{tau,sigma})^{-1} K_{tau,s}
    k = r
    C = A[:, cols[:k]] @ np.linalg.solve(A[np.ix_(rows[:k], cols[:k])], A[rows[:k], :])
    assert np.linalg.norm(C - A) <= 1e-11 * np.linalg.norm(A)


def test_aca_interpolates_pivot_rows_and_columns():
    P = inputs.points(400, 2, 9)
    I = np.flatnonzero(P[:, 0] < -0.6)
    J = np.flatnonzero(P[:, 0] > 0.3)
    K = kernels.block("log2d", P, I, J)
    rows, cols, U, V = aca.aca("log2d", P, I, J, 1e-6)
    A = U @ V.T
    assert np.allclose(A[rows, :], K[rows, :], rtol=0, atol=1e-12 * np.abs(K).max())
    assert np.allclose(A[:, cols], K[:, cols], rtol=0, atol=1e-12 * np.abs(K).max())
    # the approximation is no better than the best rank-k one (Eckart-Young) ...
    s = np.linalg.svd(K, compute_uv=False)
    k = len(rows)
    err2 = np.linalg.norm(K - A, 2)
    assert err2 >= s[k] * (1 - 1e-9)
    # ... and reaches the requested tolerance up to a modest factor
    assert np.linalg.norm(K - A) <= 100 * 1e-6 * np.linalg.norm(K)


def test_aca_rank_monotone_in_eps_and_edge_cases():
    P = inputs.points(500, 3, 13)
    I = np.flatnonzero(P[:, 2] < -0.5)
    J = np.flatnonzero(P[:, 2] > 0.2)
    ranks = [len(aca.aca("invr", P, I, J, e)[0]) for e in (1e-2, 1e-4, 1e-6, 1e-8, 1e-10)]
    assert all(a <= b for a, b in zip(ranks, ranks[1:])) and ranks[0] < ranks[-1]
    assert aca.aca("invr", P, I[:0], J, 1e-6)[0] == []
    assert len(aca.aca("invr", P, I[:3], J, 1e-16)[0]) <= 3           # rank <= min(|I|,|J|)
    Z = np.zeros((5, 7))
    assert aca.aca_entries(lambda i: Z[i], lambda j: Z[:, j], 5, 7, 1e-8)[0] == []


# --------------------------------------------------------------------------- H2 operators
@pytest.fixture(scope="module")
def h2star_small():
    P = inputs.points(1200, 2, 21)
    return h2.H2(P, "log2d", n_max=16, eps=1e-8, symmetric=False)


def test_operators_interpolate_on_pivots(h2star_small):
    """L2P U_X restricted to the rows t^{X,i} is the identity; P2M V_X^* restricted
    to the columns s^{X,o} is the identity (§3.6.4, L2P / P2M operators)."""
    H = h2star_small
    t = H.tree
    for b in H.bases.values():
        for X in range(t.nboxes(t.kappa)):
            tX = list(t.points(t.kappa, X))
            ti = b.ti[(t.kappa, X)]
            pos = [tX.index(i) for i in ti]
            k = len(ti)
            assert np.allclose(b.U[X][pos, :], np.eye(k), atol=1e-9)
            so = b.so[(t.kappa, X)]
            pos = [tX.index(i) for i in so]
            assert np.allclose(b.Vs[X][:, pos], np.eye(k), atol=1e-9)


def test_b2t_pivots_are_nested(h2star_small):
    """B2T: t^{X,i} is drawn from the union of the children's t^{X_c,i} (§5.1.1)."""
    H = h2star_small
    t, b = H.tree, H.bases["far"]
    for l in range(2, t.kappa):
        for X in range(t.nboxes(l)):
            kids = set(np.concatenate([b.ti[(l + 1, c)] for c in t.children(X)]).tolist())
            assert set(b.ti[(l, X)].tolist()) <= kids


def test_symmetric_reading_gives_transposed_operators(h2star_small):
    """With t^{X,o} = s^{X,i} and s^{X,o} = t^{X,i}: V_X = U_X, M2M = L2L^T and
    T_{Y,X} = T_{X,Y}^T (Remark after §3.6.4), so K~ is symmetric."""
    H = h2star_small
    t = H.tree

    def close(A, B, l, X, b):
        # both sides apply the inverse of the same pivot matrix in different
        # orders: rounding differences scale with its condition number
        P = H.K(b.ti[(l, X)], b.si[(l, X)])
        if P.size == 0 or A.size == 0:
            return A.shape == B.shape
        tol = 1e-14 * np.linalg.cond(P) * max(1.0, np.abs(A).max() if A.size else 0.0)
        return np.abs(A - B).max() <= tol

    for b in H.bases.values():
        for X in range(t.nboxes(t.kappa)):
            assert close(b.Vs[X], b.U[X].T, t.kappa, X, b)
        for (l1, c), Ut in b.Ut.items():
            assert close(b.Vt[(l1, c)], Ut.T, l1 - 1, c >> t.d, b)
        for (l, X, Y), T in b.T.items():
            assert np.array_equal(b.T[(l, Y, X)], T.T)
    rng = np.random.default_rng(0)
    a, c = rng.standard_normal(1200), rng.standard_normal(1200)
    assert abs(a @ H.matvec(c) - c @ H.matvec(a)) <= 1e-9 * np.linalg.norm(a) * \
        np.linalg.norm(H.matvec(c))


@pytest.mark.parametrize("variant", ["h2star", "h2plush", "h2sqrt", "h2star_t", "h2sqrt_t"])
def test_traversal_equals_assembled_matrix(variant):
    """The MVP traversal equals K~ q with K~ written out block by block from the
    same operators (separates traversal mistakes from compression error)."""
    P = inputs.points(700, 2, 31)
    H = h2.H2(P, "log2d", variant=variant, n_max=12, eps=1e-6)
    q = inputs.rhs(700, 1, 32)
    A = H.dense()
    phi = H.matvec(q)
    assert np.linalg.norm(phi - A @ q) <= 1e-13 * np.linalg.norm(A @ q)
    Q = inputs.rhs(700, 3, 33)
    assert np.allclose(H.matvec(Q), A @ Q, rtol=0, atol=1e-12 * np.abs(A @ Q).max())


@pytest.mark.parametrize("variant", ["h2star", "h2plush", "h2sqrt", "h2star_t", "h2sqrt_t"])
@pytest.mark.parametrize("kind,d", [("log2d", 2), ("invr", 3)])
def test_tight_tolerance_matches_dense(variant, kind, d):
    """At eps = 1e-12 the compressed product matches the plain definition to 1e-10."""
    N = 900 if d == 2 else 1100
    P = inputs.points(N, d, 41)
    q = inputs.rhs(N, 1, 42)
    H = h2.H2(P, kind, variant=variant, n_max=16, eps=1e-12)
    assert dense.relative_error(H.matvec(q), dense.product(kind, P, q)) <= 1e-10


def test_error_falls_with_tolerance_and_matches_paper_order():
    P = inputs.points(2500, 2, 51)
    q = inputs.rhs(2500, 1, 52)
    ex = dense.product("log2d", P, q)
    errs = []
    for eps in (1e-4, 1e-6, 1e-8, 1e-10, 1e-12):
        H = h2.H2(P, "log2d", n_max=32, eps=eps)
        errs.append(dense.relative_error(H.matvec(q), ex))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    # the paper's H2*(b+t) rows at the smallest N of each table (102400 in 2D,
    # 64000 in 3D) have RE_MVP / eps between 0.8 and 7.7; within a factor 3 of that
    rows = _golden("paper_re_mvp.txt")
    nmin = {d: min(int(r[2]) for r in rows if r[0] == d) for d in ("2", "3")}
    ratios = [float(r[3]) / float(r[1]) for r in rows if int(r[2]) == nmin[r[0]]]
    lo, hi = min(ratios), max(ratios)
    assert 0.7 < lo and hi < 8
    for e, eps in zip(errs, (1e-4, 1e-6, 1e-8, 1e-10, 1e-12)):
        assert lo / 3 <= e / eps <= 3 * hi


def test_oracle_accuracy_at_the_papers_mvp_configurations():
    """RE_MVP of the oracle's H2*(b+t) at two configurations of the paper's MVP
    tables, as written by tests/golden/make_paper_configs.py (oracle only),
    against the values the paper prints (§6.1.1, §6.2.1).  3D 1/r, n_max 125,
    N = 64000, eps 1e-6: within a factor 3 of the paper's 1.69e-6.  2D log r,
    n_max 100, N = 102400, eps 1e-8: the paper prints 1.82e-8 and the oracle
    reaches 2.2e-7; no reading of the ACA stopping rule tried closes that gap
    (they are listed with their errors in the design notes), so this bound only
    guards against the error growing further."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "oracle_re_paper_configs.txt"))
            if l.strip() and not l.startswith("#")]
    got = {(int(r[0]), int(r[2])): (float(r[6]), float(r[7])) for r in rows}
    paper = {(int(r[0]), int(r[2])): float(r[3]) for r in _golden("paper_re_mvp.txt")
             if (r[0], r[1]) in (("2", "1e-8"), ("3", "1e-6"))}
    re3, p3 = got[(3, 64000)]
    assert p3 == paper[(3, 64000)]
    assert p3 / 3 <= re3 <= 3 * p3
    re2, p2 = got[(2, 102400)]
    assert p2 == paper[(2, 102400)]
    assert re2 <= 15 * p2


def test_h2sqrt_near_field_is_larger():
    """H2_sqrt(d) does 3^d dense blocks per leaf, H2* 3^d - 2^d (Remark 3.1)."""
    P = inputs.points(2000, 3, 61)
    t = tree.Tree(P, n_max=8)
    K = t.kappa
    inner = [X for X in range(t.nboxes(K))
             if all(0 < c < (1 << K) - 1 for c in tree.key_to_coords(X, K, 3))]
    assert all(len(t.near_sqrt(K, X)) == 27 and len(t.near_star(K, X)) == 19 for X in inner)


# --------------------------------------------------------------------------- GMRES
def test_gmres_matches_dense_solve_and_residual_monotone():
    P = inputs.points(600, 2, 71)
    A = np.eye(600) + dense.matrix("log2d", P) / 600.0
    b = inputs.rhs(600, 1, 72)
    x, hist, it = gmres.gmres(lambda v: A @ v, b, rtol=1e-12, maxit=100)
    xr = gmres.dense_solve(A, b)
    assert np.linalg.norm(x - xr) <= 1e-10 * np.linalg.norm(xr)
    assert np.linalg.norm(b - A @ x) <= 1e-11 * np.linalg.norm(b)
    assert all(h1 <= h0 * (1 + 1e-12) for h0, h1 in zip(hist, hist[1:]))
    assert hist[-1] < 1e-12 and it < 100


def test_gmres_with_compressed_operator_re_sol():
    """RE_sol = ||lambda - q|| / ||q|| with b = K q and the MVP by K~ (§6)."""
    P = inputs.points(1500, 2, 81)
    q = inputs.rhs(1500, 1, 82)
    H = h2.H2(P, "log2d", n_max=32, eps=1e-10)
    op = lambda v: v + H.matvec(v) / 1500.0
    b = q + dense.product("log2d", P, q) / 1500.0
    x, hist, it = gmres.gmres(op, b, rtol=1e-12, maxit=100)
    assert np.linalg.norm(x - q) / np.linalg.norm(q) < 1e-8


@pytest.mark.parametrize("kind,d,n,eps,rtol", [("log2d", 2, 32, 1e-10, 1e-12),
                                              ("invr", 3, 8, 1e-6, 1e-10)])
def test_integral_equation_re_sol_on_the_collocation_grid(kind, d, n, eps, rtol):
    """The second-kind integral equations of §6 on the uniform collocation
    grid, (I + s K) sigma = f with s = -h^2/(2 pi) (2D, -(1/2pi) log r) or
    h^3/(4 pi) (3D, 1/(4 pi r)): with b = K q the exact solution is q, and the
    compressed solve stays within eps + 10 eps_GMRES of it."""
    P = inputs.uniform_grid(n, d)
    N = len(P)
    h = 2.0 / n
    s = -h ** 2 / (2 * math.pi) if d == 2 else h ** 3 / (4 * math.pi)
    q = inputs.rhs(N, 1, 811)
    b = q + s * dense.product(kind, P, q)
    assert np.linalg.norm(b - q) < 0.1 * np.linalg.norm(q)
    H = h2.H2(P, kind, n_max=16 if d == 2 else 8, eps=eps)
    x, hist, it = gmres.gmres(lambda v: v + s * H.matvec(v), b, rtol=rtol, maxit=200)
    assert hist[-1] < rtol
    assert np.linalg.norm(x - q) / np.linalg.norm(q) <= eps + 10 * rtol
    # the same system solved densely returns q to rounding
    xd = gmres.dense_solve(np.eye(N) + s * dense.matrix(kind, P), b)
    assert np.linalg.norm(xd - q) <= 1e-13 * np.linalg.norm(q)


def test_b2t_over_the_weak_admissibility_loses_accuracy_and_t2b_does_not():
    """§4's central observation, reproduced at a small size: with far-field and
    vertex-sharing clusters both admissible, B2T NCA over the whole list leaves
    a matrix error many orders of magnitude above eps, T2B NCA (H2*(t)) stays
    at eps, and the proposed H2*(b+t) (B2T far field, T2B vertex-sharing) too.
    The paper's values (1/r, N = 160000, n_max = 400) are in
    tests/golden/paper_b2t_vs_t2b.txt: a gap of 6 orders at eps = 1e-10; here
    2D, N = 4096, n_max = 32 (Frobenius norm, to keep the test cheap)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_b2t_vs_t2b.txt"))
            if l.strip() and not l.startswith("#")]
    paper = {float(r[0]): (float(r[1]), float(r[2])) for r in rows}
    eps = 1e-10
    assert paper[eps][0] / paper[eps][1] > 1e5
    P = inputs.points(4096, 2, 77)
    K = dense.matrix("invr", P)
    nK = np.linalg.norm(K)
    re = {v: np.linalg.norm(K - h2.H2(P, "invr", variant=v, n_max=32, eps=eps).dense()) / nK
          for v in ("h2star_b", "h2star_t", "h2star")}
    assert re["h2star_t"] <= 10 * eps
    assert re["h2star"] <= 100 * eps
    assert re["h2star_b"] >= 1e4 * re["h2star_t"]
    assert re["h2star_b"] >= 1e3 * re["h2star"]


def test_log_and_exp_are_the_c_librarys():
    """Reading of the kernels' elementary functions: log r and exp(-r) are the
    platform C library's, entry by entry (Python's math.log / math.exp call
    that library), so ACA ties on tensor grids break on the same values as in
    any C or C++ construction built on it; the other kernels use only IEEE
    operations.  A vectorised exp (numpy's on x86) differs from the C
    library's in the last bit on a few percent of these arguments, which would
    fail the equality below."""
    r = np.random.default_rng(97).uniform(1e-3, 4.0, 20000)
    assert np.array_equal(kernels.G("log2d", r), np.array([math.log(x) for x in r]))
    assert np.array_equal(kernels.G("matern12", r), np.array([math.exp(-x) for x in r]))
    P = inputs.chebyshev_grid(6, 2)
    B = kernels.block("matern12", P, np.arange(36), np.arange(36))
    for i in range(36):
        for j in range(36):
            dx, dy = P[i, 0] - P[j, 0], P[i, 1] - P[j, 1]
            want = 1.0 if i == j else math.exp(-math.sqrt(dx * dx + dy * dy))
            assert B[i, j] == want


def _clustered(d):
    """Uniform points in [-1, 1]^d plus a denser cluster in [0, side]^d (2D:
    1500 + 300 in side 0.3, strict depth 5 against the formula's 3; 3D: 1850 +
    150 in side 0.5, depth 3 against 2)."""
    nu, nc, side = (1500, 300, 0.3) if d == 2 else (1850, 150, 0.5)
    return np.vstack([inputs.points(nu, d, 801 + d), inputs.points(nc, d, 811 + d, lo=0.0, hi=side)])


def _max_occupancy(P, lo, side, k):
    c = np.clip(np.floor((P - lo) / side * float(1 << k)).astype(np.int64), 0, (1 << k) - 1)
    return int(np.unique(c, axis=0, return_counts=True)[1].max())


@pytest.mark.parametrize("d", [2, 3])
def test_strict_tree_depth_is_the_smallest_that_separates(d):
    """The strict reading of §3.1 (subdivide until every leaf holds at most
    n_max points): the depth holds every leaf to n_max, one level less does
    not (or it is the formula's depth), and on uniform points that the formula
    already separates it equals the formula's depth.  Coincident points beyond
    n_max have no such depth."""
    n_max = 32
    P = _clustered(d)
    T = tree.Tree(P, n_max=n_max, kappa="strict")
    k0 = tree.kappa_formula(P.shape[0], n_max, d)
    assert T.kappa > k0
    assert _max_occupancy(P, T.lo, T.side, T.kappa) <= n_max
    assert _max_occupancy(P, T.lo, T.side, T.kappa - 1) > n_max
    assert int(np.bincount(T.leaf_key).max()) <= n_max
    G = inputs.uniform_grid(8, d)           # 8^d points, one per box of an 8^d grid
    TG = tree.Tree(G, n_max=1, kappa="strict")
    assert TG.kappa == tree.kappa_formula(G.shape[0], 1, d) == 3
    with pytest.raises(ValueError):
        tree.Tree(np.repeat(inputs.points(4, d, 5), 40, axis=0), n_max=32, kappa="strict")
