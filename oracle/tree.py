"""The 2^d uniform tree and its interaction lists (oracle, fp64).

Tree (§3.1): level 0 is the hyper-cube C; every box of level l splits into
2^d boxes of level l+1; the leaves sit at level kappa with
kappa = ceil(log_{2^d}(N / n_max)) -- the smallest kappa with
n_max * 2^(d kappa) >= N (reading: the formula of §3.1, not "deepen until every
leaf holds <= n_max points"; that other reading is available as
kappa="strict", `kappa_strict`).

Reading of the domain C (§3.1 only asks for a compact hyper-cube holding the
points): the tight bounding cube, lo_k = min_i x_ik and side = max_k
(max_i x_ik - min_i x_ik), unless the caller passes (lo, side).  A point's box
at level kappa is floor((x - lo) / side * 2^kappa), clamped to 2^kappa - 1;
coarser boxes follow by dropping low bits, so the boxes nest exactly.

Box numbering (reading; Fig. 1's counter-clockwise numbering only orders
boxes): bit-interleaved (Morton) keys, x fastest:
key = sum_b sum_k bit_b(c_k) << (b d + k); the children of key m are
m 2^d + c, c = 0 .. 2^d - 1.  A cluster's points are listed in tree order:
by leaf key, then by original index.  All lists of clusters are in
ascending key order.

Neighbour classes (notation table of §5): two boxes of one level with integer coordinates
a, b and delta = |a - b| are
  self       if max(delta) == 0,
  far-field  F    if max(delta) >= 2 (at least one box apart),
  HS_d'      if max(delta) == 1 and exactly d' coordinates are equal
             (HS_0: vertex-sharing; HS_1: edge; HS_2 in 3D: face).
Weak admissibility (§3.5 and the notation table of §5):
  N_*(C)   = C  plus  HS_1 .. HS_{d-1}(C)                       (near field)
  clan(C)  = children of N_*(parent(C)), without C itself
             (reading: the §5 notation table writes HS_0 .. HS_{d-1} of the parent, the
             2D text of §3.5 writes its edge neighbours; only the near-field
             reading gives the maxima 12/3 (2D) and 126/7 (3D) the paper states)
  IL_far(C) = clan(C) ∩ F(C),  IL_ver(C) = clan(C) ∩ HS_0(C)   (§5.1, Fig. 6)
Strong admissibility with eta = sqrt(d) (§3.3): boxes of one level are
admissible iff they are at least one box apart, so
  N_sqrt(C)  = boxes with max(delta) <= 1 (3^d of them, self included),
  IL_sqrt(C) = children of N_sqrt(parent(C)) that are far from C.
"""

import itertools

import numpy as np


def kappa_formula(N, n_max, d):
    """Smallest kappa >= 0 with n_max * 2^(d kappa) >= N (§3.1)."""
    k = 0
    while n_max * (1 << (d * k)) < N:
        k += 1
    return k


def kappa_strict(P, n_max, lo, side, cap=20):
    """The other reading of §3.1's stopping rule ("subdivide until every leaf
    holds at most n_max points"): the smallest kappa, from the formula's up,
    at which every leaf box of the uniform tree holds at most n_max points.
    Raises ValueError when kappa would exceed `cap` (more than n_max points
    that no box size separates, e.g. coincident points)."""
    P = np.asarray(P, dtype=np.float64)
    N, d = P.shape
    k = kappa_formula(N, n_max, d)
    while True:
        c = np.clip(np.floor((P - lo) / side * float(1 << k)).astype(np.int64), 0, (1 << k) - 1)
        _, counts = np.unique(c, axis=0, return_counts=True)
        if counts.max() <= n_max:
            return k
        k += 1
        if k > cap:
            raise ValueError("no tree depth up to %d separates the points into leaves of %d" % (cap, n_max))


def bounding_cube(P):
    lo = P.min(axis=0)
    side = float((P.max(axis=0) - lo).max())
    if side <= 0.0:
        side = 1.0
    return lo, side


def morton_key(coords, level, d):
    """Bit-interleaved key of integer box coordinates (last axis = dim)."""
    coords = np.asarray(coords, dtype=np.int64)
    key = np.zeros(coords.shape[:-1], dtype=np.int64)
    for b in range(level):
        for k in range(d):
            key |= ((coords[..., k] >> b) & 1) << (b * d + k)
    return key


def key_to_coords(key, level, d):
    c = [0] * d
    for b in range(level):
        for k in range(d):
            c[k] |= ((key >> (b * d + k)) & 1) << b
    return tuple(c)


def classify(a, b):
    """'self', 'far', 'ver' (HS_0) or 'near' (HS_d', d' >= 1)."""
    delta = [abs(x - y) for x, y in zip(a, b)]
    m = max(delta)
    if m == 0:
        return "self"
    if m >= 2:
        return "far"
    n_equal = sum(1 for x in delta if x == 0)
    return "ver" if n_equal == 0 else "near"


class Tree:
    def __init__(self, P, n_max=64, kappa=None, domain=None):
        P = np.asarray(P, dtype=np.float64)
        self.P = P
        self.N, self.d = P.shape
        self.lo, self.side = bounding_cube(P) if domain is None else domain
        self.lo = np.asarray(self.lo, dtype=np.float64)
        if kappa is None:
            self.kappa = kappa_formula(self.N, n_max, self.d)
        elif kappa == "strict":
            self.kappa = kappa_strict(P, n_max, self.lo, self.side)
        else:
            self.kappa = int(kappa)
        scale = float(1 << self.kappa)
        c = np.floor((P - self.lo) / self.side * scale).astype(np.int64)
        self.leaf_coords = np.clip(c, 0, (1 << self.kappa) - 1)
        self.leaf_key = morton_key(self.leaf_coords, self.kappa, self.d)
        # tree order: by leaf key, then original index
        self.order = np.lexsort((np.arange(self.N), self.leaf_key))
        self._sorted_keys = self.leaf_key[self.order]

    # ---- clusters -------------------------------------------------------
    def nboxes(self, level):
        return 1 << (self.d * level)

    def points(self, level, key):
        """t^X of box `key` at `level`: global indices in tree order."""
        shift = self.d * (self.kappa - level)
        lo = np.searchsorted(self._sorted_keys, key << shift, side="left")
        hi = np.searchsorted(self._sorted_keys, (key + 1) << shift, side="left")
        return self.order[lo:hi]

    def children(self, key):
        return [key * (1 << self.d) + c for c in range(1 << self.d)]

    # ---- neighbour classes ------------------------------------------------
    def _boxes_around(self, level, key, radius):
        c = key_to_coords(key, level, self.d)
        n = 1 << level
        out = []
        for off in itertools.product(range(-radius, radius + 1), repeat=self.d):
            b = tuple(x + o for x, o in zip(c, off))
            if all(0 <= x < n for x in b):
                out.append(int(morton_key(b, level, self.d)))
        return sorted(out)

    def near_star(self, level, key):
        """N_*(C): self and the boxes sharing a d'-surface, d' >= 1 (§5 notation table)."""
        c = key_to_coords(key, level, self.d)
        return [b for b in self._boxes_around(level, key, 1)
                if classify(c, key_to_coords(b, level, self.d)) in ("self", "near")]

    def near_sqrt(self, level, key):
        """N_sqrt(C): the 3^d boxes at most one box away, self included (§3.3)."""
        return self._boxes_around(level, key, 1)

    def clan(self, level, key):
        if level == 0:
            return []
        parent = key >> self.d
        out = []
        for p in self.near_star(level - 1, parent):
            out.extend(ch for ch in self.children(p) if ch != key)
        return sorted(out)

    def il_far(self, level, key):
        c = key_to_coords(key, level, self.d)
        return [y for y in self.clan(level, key)
                if classify(c, key_to_coords(y, level, self.d)) == "far"]

    def il_ver(self, level, key):
        c = key_to_coords(key, level, self.d)
        return [y for y in self.clan(level, key)
                if classify(c, key_to_coords(y, level, self.d)) == "ver"]

    def il_star(self, level, key):
        """IL_*(C) = IL_far(C) u IL_ver(C): the clan members that are far-field or
        vertex-sharing (§3.5), in the clan's (ascending key) order."""
        c = key_to_coords(key, level, self.d)
        return [y for y in self.clan(level, key)
                if classify(c, key_to_coords(y, level, self.d)) in ("far", "ver")]

    def il_sqrt(self, level, key):
        if level == 0:
            return []
        c = key_to_coords(key, level, self.d)
        out = []
        for p in self.near_sqrt(level - 1, key >> self.d):
            for ch in self.children(p):
                if classify(c, key_to_coords(ch, level, self.d)) == "far":
                    out.append(ch)
        return sorted(out)
