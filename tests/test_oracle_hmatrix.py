"""Pins of the oracle's cluster tree, eq. 7 partition, ACA and half storage.

Brute force on small meshes: the partition must cover every (i, j) entry of
the matrix exactly once (counting the mirrored half), every stored far pair
must satisfy eq. 7 while its parent does not, and the compressed operator
must equal the dense Galerkin matrix up to the ACA tolerance.
"""

import numpy as np
import pytest

from oracle.hmatrix import ClusterTree, HMatrix, admissible, partition, recompress


@pytest.fixture(scope="module")
def hm_binary(sphere_small):
    # binary tree, leaf 32, eta = 1 (c = 1): far blocks at two levels
    return HMatrix(sphere_small, leaf_size=32, arity=2, adm=1.0, aca_tol=1e-4)


def test_tree_structure(sphere_small):
    m = sphere_small
    for arity, leaf in ((2, 32), (8, 32), (8, 64), (4, 100)):
        t = ClusterTree(m.centres(), *m.support_boxes(), leaf, arity)
        assert sorted(t.perm.tolist()) == list(range(m.ne))
        for d, lv in enumerate(t.levels):
            offs = [o for o, _ in lv]
            sizes = [n for _, n in lv]
            assert offs[0] == 0 and sum(sizes) == m.ne
            assert all(offs[i] + sizes[i] == offs[i + 1] for i in range(len(lv) - 1))
            assert len(lv) == arity ** d
            assert max(sizes) - min(sizes) <= 1          # median splits stay balanced
        assert max(n for _, n in t.leaves()) <= leaf
        assert t.depth == 0 or max(n for _, n in t.levels[-2]) > leaf
        for d, ch in enumerate(t.children):
            for c, kids in enumerate(ch):
                o, n = t.levels[d][c]
                assert t.levels[d + 1][kids[0]][0] == o
                assert sum(t.levels[d + 1][k][1] for k in kids) == n


def test_single_leaf_tree(sphere_tiny):
    m = sphere_tiny
    t = ClusterTree(m.centres(), *m.support_boxes(), m.ne, 8)
    assert t.depth == 0 and t.leaves() == [(0, m.ne)]
    assert partition(t, 2.0) == ([], {})


def test_partition_covers_matrix_once(sphere_small):
    m = sphere_small
    for arity, leaf, c in ((2, 32, 1.0), (8, 32, 1.0), (8, 32, 2.0), (2, 16, 0.5)):
        t = ClusterTree(m.centres(), *m.support_boxes(), leaf, arity)
        near, far = partition(t, c)
        cover = np.zeros((m.ne, m.ne), dtype=np.int32)
        for (o, n) in t.leaves():
            cover[o:o + n, o:o + n] += 1
        for (a, b) in near:
            assert a < b
            (io, mm), (jo, nn) = t.leaves()[a], t.leaves()[b]
            cover[io:io + mm, jo:jo + nn] += 1
            cover[jo:jo + nn, io:io + mm] += 1
        for d, pairs in far.items():
            for (a, b) in pairs:
                assert a < b
                (io, mm), (jo, nn) = t.levels[d][a], t.levels[d][b]
                cover[io:io + mm, jo:jo + nn] += 1
                cover[jo:jo + nn, io:io + mm] += 1
        assert cover.min() == 1 and cover.max() == 1


def test_partition_admissibility(sphere_small):
    m = sphere_small
    t = ClusterTree(m.centres(), *m.support_boxes(), 32, 2)
    near, far = partition(t, 1.0)
    parent = [dict() for _ in t.levels]
    for d, ch in enumerate(t.children):
        for c, kids in enumerate(ch):
            for k in kids:
                parent[d + 1][k] = c
    for d, pairs in far.items():
        for (a, b) in pairs:
            assert admissible(t, d, a, b, 1.0)
            if d > 0:
                pa, pb = parent[d][a], parent[d][b]
                assert pa == pb or not admissible(t, d - 1, pa, pb, 1.0)
    L = t.depth
    for (a, b) in near:
        assert not admissible(t, L, a, b, 1.0)
    # boxes: dist 0 (touching supports) is never admissible
    assert not admissible(t, L, 0, 0, 0.0)


def test_aca_and_recompression_error(sphere_small, hm_binary):
    H = hm_binary
    P = H.perm
    tol = 1e-4
    checked = 0
    for lev, blocks in H.far.items():
        for (io, mm, jo, nn, U, V) in blocks[::7]:
            Zb = sphere_small.fill(P[io:io + mm], P[jo:jo + nn])
            Ua, Va = sphere_small.aca(P[io:io + mm], P[jo:jo + nn], tol)
            err_aca = np.linalg.norm(Ua @ Va - Zb) / np.linalg.norm(Zb)
            err_rc = np.linalg.norm(U @ V - Zb) / np.linalg.norm(Zb)
            assert err_aca < 5 * tol, err_aca
            assert err_rc < 5 * tol, err_rc
            assert U.shape[1] <= Ua.shape[1]
            assert Ua.shape[1] < min(mm, nn)          # it is a low-rank block
            checked += 1
    assert checked > 10


def test_recompress_exact_low_rank():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(40, 5)) + 1j * rng.normal(size=(40, 5))
    B = rng.normal(size=(5, 30)) + 1j * rng.normal(size=(5, 30))
    # a redundant rank-10 factorisation of a rank-5 matrix
    R = rng.normal(size=(5, 5))
    U = np.concatenate([A, A @ R], axis=1)
    V = np.concatenate([0.5 * B, 0.5 * np.linalg.solve(R, B)], axis=0)
    Un, Vn = recompress(U, V, 1e-12)
    assert Un.shape[1] == 5
    assert np.linalg.norm(Un @ Vn - A @ B) < 1e-12 * np.linalg.norm(A @ B)


def test_hmatrix_matches_dense(sphere_small, dense_small, hm_binary):
    H = hm_binary
    P = H.perm
    Zt = dense_small[np.ix_(P, P)]
    # half storage: the stored operator mirrors the upper half
    iu = np.triu_indices(H.N, 1)
    Zh = Zt.copy()
    Zh[(iu[1], iu[0])] = Zt[iu]
    A = H.dense()
    assert np.linalg.norm(A - Zh) / np.linalg.norm(Zh) < 1e-4
    assert np.linalg.norm(A - A.T) / np.linalg.norm(A) < 1e-14
    # leaf-level-only operator misses exactly the coarse far blocks
    A1 = H.dense(levels=1)
    for (io, mm, jo, nn, U, V) in H.far[2]:
        assert np.all(A1[io:io + mm, jo:jo + nn] == 0)
        assert np.allclose(A[io:io + mm, jo:jo + nn], U @ V, rtol=0, atol=1e-12 * np.abs(U @ V).max())


def test_permutation_round_trip(hm_binary):
    H = hm_binary
    v = np.arange(H.N) + 0.5j
    assert np.array_equal(H.from_tree(H.to_tree(v)), v)
