"""Degenerate V-EFIE inputs on the GPU path:
- a single tetrahedron (four boundary faces, one leaf): the series has no
  coupling term, so any K gives D^{-1} b, which must equal the oracle's dense
  solve (within complex64 rounding);
- two tetrahedra sharing a face (7 unknowns, one interior): the same;
- a body whose permittivity is 1 everywhere: the contrast kappa = 1 - 1/eps_r
  vanishes, the kappa-weighted matrix is identically zero, and the leaf
  factorisation reports HM_ERR_SINGULAR instead of returning values.
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


TET = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [0.0, 0.1, 0.0], [0.0, 0.0, 0.1]])


@pytest.mark.parametrize("case", ["one_tet", "two_tets"])
def test_tiny_meshes_solve_exactly(torch_cuda, case):
    from oracle.swg import SWGMesh
    from paper_2307_03968_gb300.hm import HMatrix
    if case == "one_tet":
        xyz, tet, eps = TET, np.array([[0, 1, 2, 3]]), np.array([3.0])
    else:
        xyz = np.vstack([TET, [[0.1, 0.1, 0.1]]])
        tet, eps = np.array([[0, 1, 2, 3], [1, 2, 3, 4]]), np.array([3.0, 5.0])
    m = SWGMesh(xyz, tet, eps)
    A = HMatrix.build(xyz, tet, eps_r=eps, leaf_size=16, arity=2, adm=1.0, aca_tol=1e-4, levels=-1)
    A.factor_leaf()
    assert A.n == m.ne == (4 if case == "one_tet" else 7)
    kh, ph = np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]])
    bt = torch_cuda.empty((1, A.n), dtype=torch_cuda.complex64, device="cuda")
    A.rhs_plane_wave(kh, ph, bt)
    b = m.rhs(kh, ph)[:, 0]
    assert np.abs(bt.cpu().numpy()[0] - b).max() <= 1e-6 * np.abs(b).max()
    Z = m.dense()
    iu = np.triu_indices(A.n, 1)
    Z[(iu[1], iu[0])] = Z[iu]                      # the half-stored (mirrored) matrix the solver uses
    ref = np.linalg.solve(Z, bt.cpu().numpy()[0].astype(np.complex128))
    for K in (0, 2, 5):
        xt = torch_cuda.empty_like(bt)
        A.solve(bt, xt, n_terms=K, n_levels=-1, refine=False)
        x = xt.cpu().numpy()[0]
        assert np.linalg.norm(x - ref) <= 1e-5 * np.linalg.norm(ref), K


def test_vacuum_body_is_reported_singular(torch_cuda):
    import synth
    from paper_2307_03968_gb300.hm import HMatrix, HmError, HM_ERR_SINGULAR
    xyz, tet = synth.cube_tets(2, 0.2)
    A = HMatrix.build(xyz, tet, eps_r=np.ones(len(tet)), leaf_size=16, arity=2, adm=1.0, aca_tol=1e-4, levels=-1)
    with pytest.raises(HmError) as e:
        A.factor_leaf()
    assert e.value.status == HM_ERR_SINGULAR
