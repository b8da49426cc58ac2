"""H2*(b+t), (H2+H)* and H2_sqrt(d)(b): construction and MVP (fp64 oracle).

Follows the paper step by step, in its notation:

* B2T NCA (bottom to top) for the far field, Algorithm 1 and §5.1.1 item 1:
  at a leaf X, I = t^X and J = U_{Y in IL_far(X)} s^Y; at a non-leaf X,
  I = U_{X_c in child(X)} t^{X_c,i} and J = U_{Y in IL_far(X)} U_{Y_c} s^{Y_c,o};
  [t^{X,i}, s^{X,i}] = ACA(I, J, eps_far) for levels kappa .. 2.
* T2B NCA (top to bottom) for vertex-sharing clusters, §5.1.1 item 2:
  I = t^X, J = U_{Y in IL_ver(X)} s^Y, plus s^{parent(X),i} when X has a
  parent with pivots (levels 2 .. kappa; level 1 is parentless).  Reading:
  J is the union over all Y with the parent pivots appended once, as the text
  of §5.1.1 states (Algorithm 2's pseudocode resets J inside the loop).
* "The other two sets of pivots in a similar fashion" (Algorithms 1-2):
  reading for a symmetric kernel with the same sources and targets --
  t^{X,o} := s^{X,i} and s^{X,o} := t^{X,i}, which is what ACA on
  K_{t~^{X,o}, s~^{X,o}} = (K_{t~^{X,i}, s~^{X,i}})^T yields with the roles of
  rows and columns exchanged.
* Operators (§3.6.4): L2P U_X = K_{t^X, s^{X,i}} (K_{t^{X,i}, s^{X,i}})^{-1};
  P2M V_X^* = (K_{t^{X,o}, s^{X,o}})^{-1} K_{t^{X,o}, s^X};
  L2L U~_{X_c X} = K_{t^{X_c,i}, s^{X,i}} (K_{t^{X,i}, s^{X,i}})^{-1};
  M2M V~_{X X_c} = (K_{t^{X,o}, s^{X,o}})^{-1} K_{t^{X,o}, s^{X_c,o}};
  M2L T_{X,Y} = K_{t^{X,i}, s^{Y,o}}.  Inverses are applied by LU with
  partial pivoting (scipy), never formed.  Reading of the notation: the MVP of
  §5.1.2 applies the p_X x p_{X_c} matrix V~_{X X_c} defined above to v_{X_c}
  (the "*" printed on it in §5.1.2 would give the wrong shape).
* MVP (§5.1.2): upward (P2M at kappa; M2M at kappa-1 .. 2 far, kappa-1 .. 1
  ver), transverse (M2L at 2 .. kappa far, 1 .. kappa ver), downward (L2L at
  2 .. kappa-1 far, 1 .. kappa-1 ver; L2P at kappa) and the direct near field
  over N_*(X) at the leaves.
* (H2+H)* (§5.2): the same far field; every vertex-sharing pair (X, Y) at
  every level 1 .. kappa gets its own ACA K_{t^X, s^Y} ~ U V^* (Algorithm 3)
  and the MVP adds U (V^* q_Y) to phi(X) (Algorithm 4).
* H2_sqrt(d)(b) (App. A): one basis from B2T NCA over IL_sqrt(X), M2L at
  levels 2 .. kappa, near field over the 3^d boxes of N_sqrt(X).

Potentials are indexed by global point indices (q[t^X]), so no permutation is
involved.  Empty clusters and empty search sets give rank-0 operators.
"""

import numpy as np
import scipy.linalg

from . import kernels
from .aca import aca
from .tree import Tree


class Basis:
    """One nested basis: pivots and operators for levels lmin .. kappa."""

    def __init__(self, name, lmin, kappa):
        self.name, self.lmin, self.kappa = name, lmin, kappa
        self.ti, self.si, self.to, self.so = {}, {}, {}, {}  # (l, key) -> indices
        self.U, self.Vs = {}, {}          # leaf L2P U_X and P2M V_X^*
        self.Ut, self.Vt = {}, {}          # (l+1, child key) -> L2L / M2M
        self.T = {}                        # (l, X, Y) -> M2L T_{X,Y}
        self.il = {}                       # (l, X) -> interaction list

    def rank(self, l, key):
        return len(self.ti.get((l, key), ()))


def _lu(A):
    return scipy.linalg.lu_factor(A) if A.size else None


def _right_inv(B, lu):
    """B A^{-1} via the LU factors of A (solve A^T X^T = B^T)."""
    if B.shape[1] == 0:
        return np.zeros(B.shape)
    return scipy.linalg.lu_solve(lu, B.T, trans=1).T


def _left_inv(lu, B):
    """A^{-1} B via the LU factors of A."""
    if B.shape[0] == 0:
        return np.zeros(B.shape)
    return scipy.linalg.lu_solve(lu, B)


class H2:
    """A compressed representation K~ of the kernel matrix of points P."""

    def __init__(self, P, kind, variant="h2star", n_max=64, eps=1e-8, eps_far=None,
                 eps_ver=None, param=0.1, kappa=None, domain=None, symmetric=True,
                 store_m2l=True):
        self.P = np.asarray(P, dtype=np.float64)
        # M2L T_{X,Y} = K_{t^{X,i}, s^{Y,o}} is a plain kernel block (§3.6.4): with
        # store_m2l=False it is evaluated when applied instead of being kept.
        self.store_m2l = store_m2l
        # Remark after §3.6.4: for a symmetric kernel matrix the P2M / M2M
        # operators are the transposes of the L2P / L2L operators.  With
        # symmetric=False they are formed from their own formulas instead.
        self.symmetric = symmetric
        self.kind, self.variant, self.param = kind, variant, param
        self.eps_far = eps if eps_far is None else eps_far
        self.eps_ver = eps if eps_ver is None else eps_ver
        self.tree = Tree(self.P, n_max=n_max, kappa=kappa, domain=domain)
        t, K = self.tree, self.tree.kappa
        self.bases = {}
        if variant in ("h2star", "h2plush"):
            self.bases["far"] = self._b2t(t.il_far, self.eps_far)
        if variant == "h2star":
            self.bases["ver"] = self._t2b(t.il_ver, self.eps_ver)
        if variant == "h2plush":
            self.lowrank = self._pure_aca(self.eps_ver)
        if variant == "h2sqrt":
            self.bases["far"] = self._b2t(t.il_sqrt, self.eps_far)
        # App. C, H2*(t): one basis from T2B NCA over the whole IL_*; App. B,
        # H2_sqrt(d)(t): one basis from T2B NCA over the strong-admissibility lists
        if variant == "h2star_t":
            self.bases["far"] = self._t2b(t.il_star, self.eps_far)
        if variant == "h2sqrt_t":
            self.bases["far"] = self._t2b(t.il_sqrt, self.eps_far)
        # §4.1: B2T NCA over the whole IL_* (levels kappa .. 1) -- the pivot
        # strategy the paper shows to lose accuracy on vertex-sharing clusters
        if variant == "h2star_b":
            self.bases["far"] = self._b2t(t.il_star, self.eps_far, lmin=1)
        if variant not in ("h2star", "h2plush", "h2sqrt", "h2star_t", "h2sqrt_t", "h2star_b"):
            raise ValueError(f"unknown variant {variant}")
        self.near = t.near_sqrt if variant in ("h2sqrt", "h2sqrt_t") else t.near_star
        for b in self.bases.values():
            self._operators(b)
        self.kappa = K

    def K(self, rows, cols):
        return kernels.block(self.kind, self.P, rows, cols, self.param)

    # ---- pivot selection --------------------------------------------------
    def _b2t(self, il, eps, lmin=2):
        """B2T NCA (Algorithm 1) over the lists `il`, levels kappa .. lmin."""
        t, K = self.tree, self.tree.kappa
        b = Basis("far", lmin, K)
        empty = np.zeros(0, dtype=np.int64)
        for l in range(K, lmin - 1, -1):
            for X in range(t.nboxes(l)):
                Ys = il(l, X)
                b.il[(l, X)] = Ys
                if l == K:
                    I = t.points(l, X)
                    J = np.concatenate([t.points(l, Y) for Y in Ys] + [empty])
                else:
                    I = np.concatenate([b.ti[(l + 1, c)] for c in t.children(X)] + [empty])
                    J = np.concatenate([b.so[(l + 1, c)] for Y in Ys for c in t.children(Y)]
                                       + [empty])
                rows, cols, _, _ = aca(self.kind, self.P, I, J, eps, self.param)
                b.ti[(l, X)] = I[np.asarray(rows, dtype=np.int64)]
                b.si[(l, X)] = J[np.asarray(cols, dtype=np.int64)]
                b.to[(l, X)] = b.si[(l, X)]
                b.so[(l, X)] = b.ti[(l, X)]
        return b

    def _t2b(self, il, eps):
        """T2B NCA (§5.1.1 item 2) over the lists `il`, levels 1 .. kappa."""
        t, K = self.tree, self.tree.kappa
        b = Basis("ver", 1, K)
        empty = np.zeros(0, dtype=np.int64)
        for l in range(1, K + 1):
            for X in range(t.nboxes(l)):
                Ys = il(l, X)
                b.il[(l, X)] = Ys
                I = t.points(l, X)
                parts = [t.points(l, Y) for Y in Ys]
                if l > 1:
                    parts.append(b.si[(l - 1, X >> t.d)])
                J = np.concatenate(parts + [empty])
                rows, cols, _, _ = aca(self.kind, self.P, I, J, eps, self.param)
                b.ti[(l, X)] = I[np.asarray(rows, dtype=np.int64)]
                b.si[(l, X)] = J[np.asarray(cols, dtype=np.int64)]
                b.to[(l, X)] = b.si[(l, X)]
                b.so[(l, X)] = b.ti[(l, X)]
        return b

    def _pure_aca(self, eps):
        """Algorithm 3: plain ACA of every vertex-sharing block, levels 1 .. kappa."""
        t, out = self.tree, {}
        self.il_ver = {}
        for l in range(1, t.kappa + 1):
            for X in range(t.nboxes(l)):
                I = t.points(l, X)
                self.il_ver[(l, X)] = t.il_ver(l, X)
                for Y in self.il_ver[(l, X)]:
                    J = t.points(l, Y)
                    _, _, U, V = aca(self.kind, self.P, I, J, eps, self.param)
                    out[(l, X, Y)] = (U, V)
        return out

    # ---- operators (§3.6.4) ---------------------------------------------------
    def _operators(self, b):
        t, K = self.tree, b.kappa
        if K < b.lmin:
            return
        lu_i, lu_o = {}, {}
        for l in range(b.lmin, K + 1):
            for X in range(t.nboxes(l)):
                lu_i[(l, X)] = _lu(self.K(b.ti[(l, X)], b.si[(l, X)]))
                lu_o[(l, X)] = _lu(self.K(b.to[(l, X)], b.so[(l, X)]))
        for X in range(t.nboxes(K)):
            tX = t.points(K, X)
            b.U[X] = _right_inv(self.K(tX, b.si[(K, X)]), lu_i[(K, X)])
            b.Vs[X] = b.U[X].T if self.symmetric else \
                _left_inv(lu_o[(K, X)], self.K(b.to[(K, X)], tX))
        for l in range(b.lmin, K):
            for X in range(t.nboxes(l)):
                for c in t.children(X):
                    b.Ut[(l + 1, c)] = _right_inv(self.K(b.ti[(l + 1, c)], b.si[(l, X)]),
                                                  lu_i[(l, X)])
                    b.Vt[(l + 1, c)] = b.Ut[(l + 1, c)].T if self.symmetric else \
                        _left_inv(lu_o[(l, X)], self.K(b.to[(l, X)], b.so[(l + 1, c)]))
        if self.store_m2l:
            for l in range(b.lmin, K + 1):
                for X in range(t.nboxes(l)):
                    for Y in b.il[(l, X)]:
                        b.T[(l, X, Y)] = self.K(b.ti[(l, X)], b.so[(l, Y)])

    # ---- the MVP (§5.1.2, §5.2.2, App. A.2) -------------------------------------
    def matvec(self, q):
        q = np.asarray(q, dtype=np.float64)
        t, K = self.tree, self.tree.kappa
        phi = np.zeros_like(q)
        for b in self.bases.values():
            phi += self._nested_potential(b, q)
        if self.variant == "h2plush":
            for (l, X, Y), (U, V) in self.lowrank.items():
                phi[t.points(l, X)] += U @ (V.T @ q[t.points(l, Y)])
        for X in range(t.nboxes(K)):
            tX = t.points(K, X)
            for Xn in self.near(K, X):
                sX = t.points(K, Xn)
                phi[tX] += self.K(tX, sX) @ q[sX]
        return phi

    def _nested_potential(self, b, q):
        t, K = self.tree, b.kappa
        phi = np.zeros_like(q)
        if K < b.lmin:
            return phi
        v, u = {}, {}
        # upward traversal: P2M at the leaves, M2M at kappa-1 .. lmin
        for X in range(t.nboxes(K)):
            v[(K, X)] = b.Vs[X] @ q[t.points(K, X)]
        for l in range(K - 1, b.lmin - 1, -1):
            for X in range(t.nboxes(l)):
                acc = np.zeros((b.rank(l, X),) + q.shape[1:])
                for c in t.children(X):
                    acc += b.Vt[(l + 1, c)] @ v[(l + 1, c)]
                v[(l, X)] = acc
        # transverse traversal: M2L at lmin .. kappa
        for l in range(b.lmin, K + 1):
            for X in range(t.nboxes(l)):
                acc = np.zeros((b.rank(l, X),) + q.shape[1:])
                for Y in b.il[(l, X)]:
                    T = b.T[(l, X, Y)] if self.store_m2l else self.K(b.ti[(l, X)], b.so[(l, Y)])
                    acc += T @ v[(l, Y)]
                u[(l, X)] = acc
        # downward traversal: L2L at lmin .. kappa-1, L2P at the leaves
        for l in range(b.lmin, K):
            for X in range(t.nboxes(l)):
                for c in t.children(X):
                    u[(l + 1, c)] = u[(l + 1, c)] + b.Ut[(l + 1, c)] @ u[(l, X)]
        for X in range(t.nboxes(K)):
            phi[t.points(K, X)] += b.U[X] @ u[(K, X)]
        return phi

    # ---- the compressed matrix written out (for checking the traversal) -------
    def full_bases(self, b):
        """U_X and V_X over all of t^X for every cluster, expanded through the
        nested L2L / M2M operators (Eqs. of the L2L and M2M operators, §3.6.4)."""
        t, K = self.tree, b.kappa
        U, V = {}, {}
        for X in range(t.nboxes(K)):
            U[(K, X)] = b.U[X]
            V[(K, X)] = b.Vs[X].T
        for l in range(K - 1, b.lmin - 1, -1):
            for X in range(t.nboxes(l)):
                ch = t.children(X)
                U[(l, X)] = np.concatenate(
                    [U[(l + 1, c)] @ b.Ut[(l + 1, c)] for c in ch], axis=0)
                V[(l, X)] = np.concatenate(
                    [V[(l + 1, c)] @ b.Vt[(l + 1, c)].T for c in ch], axis=0)
        return U, V

    def dense(self):
        """K~ as an N x N matrix assembled block by block from the operators."""
        t, K = self.tree, self.tree.kappa
        A = np.zeros((t.N, t.N))
        for b in self.bases.values():
            if K < b.lmin:
                continue
            U, V = self.full_bases(b)
            for (l, X, Y), T in b.T.items():
                A[np.ix_(t.points(l, X), t.points(l, Y))] += U[(l, X)] @ T @ V[(l, Y)].T
        if self.variant == "h2plush":
            for (l, X, Y), (Ul, Vl) in self.lowrank.items():
                A[np.ix_(t.points(l, X), t.points(l, Y))] += Ul @ Vl.T
        for X in range(t.nboxes(K)):
            for Xn in self.near(K, X):
                rX, sX = t.points(K, X), t.points(K, Xn)
                A[np.ix_(rX, sX)] += self.K(rX, sX)
        return A

    # ---- statistics -------------------------------------------------------------
    def ranks(self, name):
        b, t = self.bases[name], self.tree
        return {l: [b.rank(l, X) for X in range(t.nboxes(l))]
                for l in range(b.lmin, b.kappa + 1)}
