"""Leaves above the shared-memory factorisation (more than 112 unknowns), toward
the paper's leaf sizes (arxiv 2307.03968 §IV: binary trees to levels 6, 8 and 10,
about 1,050, 620 and 117 unknowns per leaf): the FP64 Gauss-Jordan of the large
leaves runs as batched pivot steps over a device workspace.

- the factorisation alone: the oracle's FP64 leaf self blocks (entry by entry,
  for the oracle's tree) imported as a block-diagonal operator, x = D^{-1} b with
  zero series terms against numpy's solve of the same blocks (leaves of 240 and
  960 unknowns), within the complex64 storage of D^{-1} (kappa x ~1e-7);
- the whole K = 2 leaf-level solve with refinement on 240-unknown leaves, the
  oracle's H-Matrix imported, against the oracle running the same algorithm.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03968_gb300 import build
    build.build()
    return torch


def _block_diagonal(sub, radius, leaf_size):
    import synth
    from oracle.rwg import RWGMesh
    from oracle.hmatrix import ClusterTree
    xyz, tri = synth.icosphere(sub, radius)
    mesh = RWGMesh(xyz, tri)
    lo, hi = mesh.support_boxes()
    tree = ClusterTree(mesh.centres(), lo, hi, leaf_size, arity=2)
    leaves = tree.leaves()
    D = [mesh.fill(tree.perm[o:o + n], tree.perm[o:o + n]) for (o, n) in leaves]
    leaf_off = [0] + [o + n for (o, n) in leaves]
    b = mesh.rhs(np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))[:, 0]
    return tree.perm, leaf_off, D, b


@pytest.mark.parametrize("sub,radius,leaf_size", [(3, 0.3, 300), (4, 1.0, 1000)])
def test_large_leaf_inverse(torch_cuda, sub, radius, leaf_size):
    from paper_2307_03968_gb300.hm import HMatrix
    perm, leaf_off, D, b = _block_diagonal(sub, radius, leaf_size)
    sizes = np.diff(leaf_off)
    assert sizes.min() > 112
    A = HMatrix.from_blocks(perm, leaf_off, D, [], [])
    A.factor_leaf()
    bt = torch_cuda.from_numpy(b.astype(np.complex64)).cuda()
    xt = torch_cuda.empty_like(bt)
    A.solve(bt, xt, n_terms=0, n_levels=1, refine=False)
    x = xt.cpu().numpy()
    for i, (o, n) in enumerate(zip(leaf_off[:-1], sizes)):
        rows = perm[o:o + n]
        ref = np.linalg.solve(D[i], b[rows])
        kappa = np.linalg.cond(D[i])
        err = np.linalg.norm(x[rows] - ref) / np.linalg.norm(ref)
        assert err < max(1e-5, 3e-7 * kappa), (i, n, kappa, err)
    A.close()


def test_large_leaf_solve_matches_oracle(torch_cuda):
    import synth
    from oracle.rwg import RWGMesh
    from oracle.hmatrix import HMatrix as OracleH
    from oracle import series
    from paper_2307_03968_gb300.hm import HMatrix
    xyz, tri = synth.icosphere(3, 0.3)
    mesh = RWGMesh(xyz, tri)
    H = OracleH(mesh, leaf_size=300, arity=2, adm=1.0, aca_tol=1e-4)
    assert max(n for (o, n) in H.leaves) > 112
    b = mesh.rhs(np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))[:, 0]
    ref = series.solve(H, b, K=2, levels=1, refine=True)
    leaf_off = [0] + [o + n for (o, n) in H.leaves]
    near = [(io, jo, B) for (io, m, jo, n, B) in H.near]
    far = [(lev, io, jo, U, V) for lev, lst in sorted(H.far.items()) for (io, m, jo, n, U, V) in lst]
    A = HMatrix.from_blocks(H.perm, leaf_off, H.D, near, far)
    A.factor_leaf()
    bt = torch_cuda.from_numpy(b.astype(np.complex64)).cuda()
    xt = torch_cuda.empty_like(bt)
    A.solve(bt, xt, n_terms=2, n_levels=1, refine=True)
    x = xt.cpu().numpy()
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-4
    A.close()
