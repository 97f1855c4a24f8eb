"""Cluster tree, admissibility, block partition and the half-stored H-Matrix.

Oracle — test infrastructure only.  Follows arxiv 2307.03968 §III:
  - the mesh is split by a tree "terminated ... with a limiting edge or face
    count" (§III); the paper's runs use a binary tree, an octree is the default
    here (arity 8 = three binary splits collapsed into one level);
  - eq. 7 admissibility, read as  dist(t, s) >= c * min(diam t, diam s), c = 1/eta
    (the paper's eta = 1.0 gives c = 1; the workloads use c = 2);
  - a pair is stored at the coarsest level where it is admissible and is not
    split further ("parent interaction ... not computed", §III);
  - non-admissible leaf pairs are dense near blocks (eq. 6, Z_N);
  - far blocks are compressed with ACA (refs. [22,23]) and re-compressed
    (ref. [24]: QR of both factors + SVD of the small core, truncated at tol);
  - only half of the matrix is computed, Z being complex symmetric (§III,
    ref. [12]): pairs t <= s are filled and Z[s, t] = Z[t, s]^T.

Readings where the paper is silent:
  - splitting rule: sort the cluster's unknowns by (coordinate of the edge
    midpoint along the longest axis of their bounding box, original index) and
    cut after n // 2; ties in the axis choice go to the lower axis index;
  - every cluster is split until all leaves hold at most ``leaf_size`` unknowns,
    so all leaves lie at the same depth L;
  - cluster geometry = bounding box of the vertices of the supports (T+ and T-)
    of its unknowns; dist = distance between boxes, diam = box diagonal; a pair
    with dist = 0 is never admissible.
"""

import numpy as np


class ClusterTree:
    """levels[d] = list of (offset, size) in tree order, d = 0 (root) .. L (leaves).
    ``perm[p]`` = original index of the unknown at tree position p.
    ``children[d][c]`` = indices at depth d+1 of the children of cluster c."""

    def __init__(self, centres, box_lo, box_hi, leaf_size, arity=8):
        if arity not in (2, 4, 8):
            raise ValueError("arity must be 2, 4 or 8")
        N = len(centres)
        self.N, self.arity, self.leaf_size = N, arity, leaf_size
        splits = {2: 1, 4: 2, 8: 3}[arity]
        clusters = [np.arange(N, dtype=np.int64)]
        levels_idx = [clusters]
        children = []
        while max(len(c) for c in clusters) > leaf_size:
            nxt, ch = [], []
            for c in clusters:
                parts = [c]
                for _ in range(splits):
                    parts = [half for p in parts for half in self._bisect(p, centres)]
                if any(len(p) == 0 for p in parts):
                    raise ValueError("leaf_size too small for this arity: a cluster would be empty")
                ch.append(list(range(len(nxt), len(nxt) + len(parts))))
                nxt += parts
            children.append(ch)
            clusters = nxt
            levels_idx.append(clusters)
        self.depth = len(levels_idx) - 1
        self.children = children
        self.perm = np.concatenate(levels_idx[-1]).astype(np.int64)
        pos = np.empty(N, dtype=np.int64)
        pos[self.perm] = np.arange(N)
        self.levels = []
        self.box = []
        for cl in levels_idx:
            lv, bx = [], []
            for c in cl:
                p = pos[c]
                off = int(p.min())
                assert np.array_equal(np.sort(p), np.arange(off, off + len(c)))
                lv.append((off, len(c)))
                bx.append((box_lo[c].min(axis=0), box_hi[c].max(axis=0)))
            self.levels.append(lv)
            self.box.append(bx)

    @staticmethod
    def _bisect(idx, centres):
        pts = centres[idx]
        ext = pts.max(axis=0) - pts.min(axis=0)
        axis = int(np.argmax(ext))          # first maximum = lowest axis index on ties
        order = np.lexsort((idx, pts[:, axis]))
        s = idx[order]
        h = len(s) // 2
        return [s[:h], s[h:]]

    def leaves(self):
        return self.levels[-1]


def box_dist(lo1, hi1, lo2, hi2):
    gap = np.maximum(0.0, np.maximum(lo2 - hi1, lo1 - hi2))
    return float(np.sqrt(np.sum(gap * gap)))


def box_diam(lo, hi):
    e = hi - lo
    return float(np.sqrt(np.sum(e * e)))


def admissible(tree, d, t, s, c):
    """eq. 7: c * ... read as dist >= c * min(diam); dist = 0 is never admissible."""
    lo1, hi1 = tree.box[d][t]
    lo2, hi2 = tree.box[d][s]
    dist = box_dist(lo1, hi1, lo2, hi2)
    return dist > 0.0 and dist >= c * min(box_diam(lo1, hi1), box_diam(lo2, hi2))


def partition(tree, c):
    """Half block partition.  Returns (near, far): near = [(t, s)] leaf pairs t < s
    (self pairs t == s are the leaf blocks D); far = {depth: [(t, s)]} with t < s.
    Pairs are listed in depth-first order of the recursion."""
    near, far = [], {}
    L = tree.depth

    def rec(d, t, s):
        if t != s and admissible(tree, d, t, s, c):
            far.setdefault(d, []).append((t, s))
            return
        if d == L:
            if t != s:
                near.append((t, s))
            return
        for ct in tree.children[d][t]:
            for cs in tree.children[d][s]:
                if t == s and ct > cs:
                    continue
                rec(d + 1, ct, cs)

    rec(0, 0, 0)
    return near, far


def recompress(U, V, tol):
    """Re-compressed ACA (ref. [24]): U V = Qu Ru (Qv Rv)^T; SVD of Ru Rv^T;
    keep the smallest rank r whose discarded singular values have Frobenius
    norm <= tol * (Frobenius norm of all of them)."""
    k = U.shape[1]
    if k == 0:
        return U, V
    Qu, Ru = np.linalg.qr(U)
    Qv, Rv = np.linalg.qr(V.T)
    W, sig, Zh = np.linalg.svd(Ru @ Rv.T)
    tail = np.sqrt(np.cumsum((sig ** 2)[::-1]))[::-1]   # tail[i] = |sig[i:]|
    total = tail[0]
    r = k
    for i in range(1, k + 1):
        if i == k or tail[i] <= tol * total:
            r = i
            break
    Un = Qu @ (W[:, :r] * sig[:r])
    Vn = Zh[:r, :] @ Qv.T
    return Un, Vn


class HMatrix:
    """Half-stored H-Matrix of an RWG mesh in tree order (complex128).

    D[i]          dense leaf self block (n_i x n_i)
    near          [(I_off, m, J_off, n, B)] with B = Z[I, J] for leaf pairs I < J
    far[level]    [(t_off, m, s_off, n, U, V)], Z[t, s] ~ U V, level counted
                  from the leaf: level 1 = depth L, level 2 = depth L-1, ...
    """

    def __init__(self, mesh, leaf_size=32, arity=8, adm=2.0, aca_tol=1e-4,
                 levels=None, recompression=True):
        self.mesh = mesh
        self.tree = ClusterTree(mesh.centres(), *mesh.support_boxes(), leaf_size, arity)
        t = self.tree
        self.N = t.N
        self.perm = t.perm
        self.depth = t.depth
        near_pairs, far_pairs = partition(t, adm)
        self.near_pairs, self.far_pairs = near_pairs, far_pairs
        P = t.perm
        self.leaves = t.leaves()
        # leaf self blocks: fill the upper triangle (local i <= j), mirror (half storage)
        self.D = []
        for (off, n) in self.leaves:
            idx = P[off:off + n]
            B = mesh.fill(idx, idx)
            iu = np.triu_indices(n, 1)
            B[(iu[1], iu[0])] = B[iu]
            self.D.append(B)
        self.near = []
        for (a, b) in near_pairs:
            (io, m), (jo, n) = self.leaves[a], self.leaves[b]
            self.near.append((io, m, jo, n, mesh.fill(P[io:io + m], P[jo:jo + n])))
        self.far = {}
        self.n_levels = 1 + max([self.depth - d for d in far_pairs] + [0])
        for d, pairs in sorted(far_pairs.items()):
            lev = self.depth - d + 1
            if levels is not None and lev > levels:
                continue
            blocks = [(P[t.levels[d][a][0]:t.levels[d][a][0] + t.levels[d][a][1]],
                       P[t.levels[d][b][0]:t.levels[d][b][0] + t.levels[d][b][1]]) for (a, b) in pairs]
            facs = mesh.aca_many(blocks, aca_tol)
            lst = []
            for (a, b), (U, V) in zip(pairs, facs):
                if recompression:
                    U, V = recompress(U, V, aca_tol)
                (io, m), (jo, n) = t.levels[d][a], t.levels[d][b]
                lst.append((io, m, jo, n, U, V))
            self.far[lev] = lst

    # ---- operators in tree order, x of shape (N, R) ----------------------------------
    def apply_D(self, x):
        y = np.zeros_like(x)
        for (off, n), B in zip(self.leaves, self.D):
            y[off:off + n] = B @ x[off:off + n]
        return y

    def solve_D(self, x):
        """D^{-1} x by a dense LU solve of each leaf self block (eq. 12)."""
        y = np.zeros_like(x)
        for (off, n), B in zip(self.leaves, self.D):
            y[off:off + n] = np.linalg.solve(B, x[off:off + n])
        return y

    def apply_M(self, level, x):
        """M_level x.  M_1 = off-diagonal near blocks + leaf-level far blocks;
        M_l (l >= 2) = far blocks l-1 levels above the leaves.  Half storage:
        every stored block acts on both of its row clusters."""
        z = np.zeros_like(x)
        if level == 1:
            for (io, m, jo, n, B) in self.near:
                z[io:io + m] += B @ x[jo:jo + n]
                z[jo:jo + n] += B.T @ x[io:io + m]
        for (io, m, jo, n, U, V) in self.far.get(level, []):
            z[io:io + m] += U @ (V @ x[jo:jo + n])
            z[jo:jo + n] += V.T @ (U.T @ x[io:io + m])
        return z

    def apply(self, x, levels=None):
        """A_m x = D x + sum_{l <= m} M_l x (the H-Matrix truncated at m levels)."""
        m = self.n_levels if levels is None or levels < 0 else levels
        y = self.apply_D(x)
        for lev in range(1, m + 1):
            y += self.apply_M(lev, x)
        return y

    def dense(self, levels=None):
        """Dense A_m in tree order (small N only)."""
        return self.apply(np.eye(self.N, dtype=np.complex128), levels)

    # ---- permutation -----------------------------------------------------------------
    def to_tree(self, v):
        return v[self.perm]

    def from_tree(self, v):
        out = np.empty_like(v)
        out[self.perm] = v
        return out

    def stats(self):
        near = sum(m * n for (_, m, _, n, _) in self.near)
        far = {lev: sum(U.shape[1] * (m + n) for (_, m, _, n, U, _) in lst)
               for lev, lst in self.far.items()}
        dd = sum(n * n for (_, n) in self.leaves)
        return {"N": self.N, "depth": self.depth, "leaves": len(self.leaves),
                "near_blocks": len(self.near), "near_elems": near, "self_elems": dd,
                "far_blocks": {l: len(v) for l, v in self.far.items()}, "far_elems": far,
                "max_rank": {l: max([U.shape[1] for (_, _, _, _, U, _) in v] + [0])
                             for l, v in self.far.items()}}
