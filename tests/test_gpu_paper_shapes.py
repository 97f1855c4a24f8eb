"""GPU operators of small synthetic versions of the paper's experiment shapes
(arxiv 2307.03968 §IV) against the oracle: an open PEC plate (RWG functions on
interior edges only; the plate's rim carries none) and a hollow dielectric
cylinder (SWG on a periodic cylindrical-shell mesh), with the paper's settings
(binary tree, eq. 7 with eta = 1, ACA 1e-3):
- tree and partition bit-exact with the oracle's;
- the GPU-built operator's product within 5 x tol of the oracle's H-Matrix;
- the K-term series of the oracle's own operator (imported) within 1e-4 of the
  oracle's series, for K = 2 (the paper's) and K = 8.
"""

import numpy as np
import pytest

from hm_testutil import rel_err, gpu_operator

pytestmark = pytest.mark.gpu

TOL = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03968_gb300 import build
    build.build()
    return torch


def shapes():
    import synth
    xyz, tri = synth.plate((2.0, 2.0), (20, 20))                  # 1,160 RWG
    xs, ts = synth.shell_tets(0.35, 0.4, 1.2, (1, 24, 12))         # 4,080 SWG
    return {"plate": (xyz, tri, None), "hollow_cylinder": (xs, ts, np.full(len(ts), 2.0))}


@pytest.fixture(scope="module")
def built(torch_cuda):
    from oracle.rwg import RWGMesh
    from oracle.swg import SWGMesh
    from oracle.hmatrix import HMatrix as OH
    from paper_2307_03968_gb300.hm import HMatrix
    out = {}
    for name, (xyz, cells, eps) in shapes().items():
        mesh = RWGMesh(xyz, cells) if eps is None else SWGMesh(xyz, cells, eps)
        kw = dict(leaf_size=32, arity=2, adm=1.0, aca_tol=TOL)
        A = HMatrix.build(xyz, cells, eps_r=eps, levels=-1, **kw)
        A.factor_leaf()
        out[name] = (mesh, A, OH(mesh, **kw))
    return out


@pytest.mark.parametrize("name", ["plate", "hollow_cylinder"])
def test_shape_tree_and_operator(torch_cuda, built, name):
    mesh, A, H = built[name]
    assert A.n == H.N == mesh.ne
    assert np.array_equal(A.perm(), H.perm)
    assert A.info().n_levels == H.n_levels
    rng = np.random.default_rng(2)
    x = (rng.normal(size=(2, A.n)) + 1j * rng.normal(size=(2, A.n))).astype(np.complex64)
    xt = torch_cuda.from_numpy(x).cuda()
    yt = torch_cuda.empty_like(xt)
    A.apply(xt, yt, n_levels=-1, fp64_accumulate=True)
    ref = H.from_tree(H.apply(H.to_tree(x.T.astype(np.complex128)))).T
    assert rel_err(yt.cpu().numpy(), ref) < 5 * TOL


@pytest.mark.parametrize("name", ["plate", "hollow_cylinder"])
@pytest.mark.parametrize("K", [2, 8])
def test_shape_series_parity(torch_cuda, built, name, K):
    from oracle import series
    mesh, _, H = built[name]
    G = gpu_operator(H)
    kh = np.array([[0.3, 0.2, -1.0]]) / np.linalg.norm([0.3, 0.2, -1.0])
    ph = np.array([[1.0, 0.0, 0.3]]) / np.linalg.norm([1.0, 0.0, 0.3])
    b = mesh.rhs(kh, ph)
    ref = series.solve(H, b, K=K, levels=H.n_levels, nested_form=False).T
    bt = torch_cuda.from_numpy(b.T.astype(np.complex64).copy()).cuda()
    xt = torch_cuda.empty_like(bt)
    G.solve(bt, xt, n_terms=K, n_levels=-1, nested=False)
    assert rel_err(xt.cpu().numpy(), ref) < 1e-4
