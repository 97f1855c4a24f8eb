"""GPU V-EFIE (SWG basis, arxiv 2307.03968 §II eq. 4) against the oracle.

Small case: an inhomogeneous dielectric slab 2 x 0.25 x 0.125 wavelengths
(4 x 4 x 4 voxels, 384 tetrahedra, 864 SWG unknowns, eps_r iid uniform [2, 6])
whose shape leaves far blocks on several tree levels:
- tree, leaves and block partition bit-exact with the oracle's;
- near blocks filled on the device (complex64) vs the oracle's complex128
  entries: elementwise, relative to the block's largest entry, <= 2e-5 (FP32
  quadrature; the analytic singular terms are taken in FP64);
- far blocks: U V against the oracle's dense block, relative Frobenius <= 5 tol;
- leaf self blocks (FP64 fill, FP64 factorisation): D^{-1} b (a solve with no
  series term) vs the oracle's dense LU solve of each leaf, <= 1e-5;
- plane-wave right-hand sides, 16 random incidences, elementwise <= 1e-6;
- the whole operator: hm_apply vs the oracle's H-Matrix product <= 5 tol;
- the power-series solve of the oracle's own operator (imported blocks),
  leaf level and all levels, <= 1e-4 relative to the oracle's solve.

Full size: the 1-wavelength dielectric cube with 41,850 SWG unknowns (15^3
voxels, 20,250 tetrahedra, eps_r iid uniform [2, 6] from seed 4), binary tree,
leaf 64, eq. 7 with eta = 1, ACA 1e-4, 16 random incidences: sampled product
rows against the oracle's dense rows, the device RHS elementwise, and solve
reciprocity (every series term is symmetric).
"""

import numpy as np
import pytest

from hm_testutil import rel_err, gpu_operator

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03968_gb300 import build
    build.build()
    return torch


def slab_mesh():
    import synth
    xyz, tet = synth.cube_tets(4, 1.0)
    xyz = xyz * np.array([2.0, 0.25, 0.125])
    eps = synth.random_permittivity(len(tet), 2.0, 6.0, seed=4)
    return xyz, tet, eps


CASES = {
    "binary_leaf16_c1": dict(leaf_size=16, arity=2, adm=1.0),
    "octree_leaf32_c2": dict(leaf_size=32, arity=8, adm=2.0),
}


@pytest.fixture(scope="module")
def slab(torch_cuda):
    from oracle.swg import SWGMesh
    from oracle.hmatrix import HMatrix as OH
    from paper_2307_03968_gb300.hm import HMatrix
    xyz, tet, eps = slab_mesh()
    mesh = SWGMesh(xyz, tet, eps)
    out = {}
    for name, kw in CASES.items():
        A = HMatrix.build(xyz, tet, eps_r=eps, aca_tol=TOL, levels=-1, **kw)
        A.factor_leaf()
        out[name] = (A, OH(mesh, aca_tol=TOL, **kw))
    return mesh, out


@pytest.mark.parametrize("name", list(CASES))
def test_swg_tree_and_partition_bit_exact(slab, name):
    mesh, built = slab
    A, H = built[name]
    assert A.n == mesh.ne == 864
    assert np.array_equal(A.perm(), H.perm)
    assert np.array_equal(A.leaves(), [0] + [o + n for (o, n) in H.leaves])
    assert A.info().n_levels == H.n_levels
    r0, c0, m, n, k = A.blocks(1)
    dense = k == 0
    assert sorted(zip(r0[dense], c0[dense], m[dense], n[dense])) == \
        sorted((io, jo, mm, nn) for (io, mm, jo, nn, _) in H.near)
    for lev, lst in H.far.items():
        r0, c0, m, n, k = A.blocks(lev)
        lr = k > 0
        assert sorted(zip(r0[lr], c0[lr], m[lr], n[lr])) == \
            sorted((io, jo, mm, nn) for (io, mm, jo, nn, _, _) in lst), lev


@pytest.mark.parametrize("name", list(CASES))
def test_swg_near_blocks_match_oracle_fill(slab, name):
    mesh, built = slab
    A, H = built[name]
    P = H.perm
    r0, c0, m, n, k = A.blocks(1)
    worst, checked = 0.0, 0
    for idx in range(0, len(k), 7):
        if k[idx] != 0:
            continue
        B = A.block(1, idx)
        ref = mesh.fill(P[r0[idx]:r0[idx] + m[idx]], P[c0[idx]:c0[idx] + n[idx]])
        worst = max(worst, np.abs(B - ref).max() / np.abs(ref).max())
        checked += 1
    assert checked >= 10
    assert worst < 2e-5, worst


def test_swg_far_blocks_within_aca_tolerance(slab):
    mesh, built = slab
    A, H = built["binary_leaf16_c1"]
    P = H.perm
    checked = 0
    for lev in range(1, A.info().n_levels + 1):
        r0, c0, m, n, k = A.blocks(lev)
        for idx in np.nonzero(k > 0)[0][::3]:
            U, V = A.block(lev, idx)
            Zb = mesh.fill(P[r0[idx]:r0[idx] + m[idx]], P[c0[idx]:c0[idx] + n[idx]])
            err = np.linalg.norm(U @ V - Zb) / np.linalg.norm(Zb)
            assert err < 5 * TOL, (lev, idx, err, k[idx])
            assert k[idx] < min(m[idx], n[idx])
            checked += 1
    assert checked >= 8


@pytest.mark.parametrize("name", list(CASES))
def test_swg_leaf_inverses_match_oracle(torch_cuda, slab, name):
    # x = D^{-1} b (no series term): the FP64 self-block fill and factorisation
    import synth
    mesh, built = slab
    A, H = built[name]
    k, p = synth.random_incidences(4, seed=9)
    b = mesh.rhs(k, p)                                   # (N, 4)
    ref = H.from_tree(H.solve_D(H.to_tree(b))).T
    bt = torch_cuda.from_numpy(b.T.astype(np.complex64).copy()).cuda()
    xt = torch_cuda.empty_like(bt)
    A.solve(bt, xt, n_terms=0, n_levels=1, refine=False)
    assert rel_err(xt.cpu().numpy(), ref) < 1e-5


def test_swg_rhs_matches_oracle(torch_cuda, slab):
    import synth
    mesh, built = slab
    A, _ = built["binary_leaf16_c1"]
    k, p = synth.random_incidences(16, seed=21)
    bt = torch_cuda.empty((16, A.n), dtype=torch_cuda.complex64, device="cuda")
    A.rhs_plane_wave(k, p, bt)
    ref = mesh.rhs(k, p).T
    got = bt.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("name", list(CASES))
def test_swg_operator_matches_oracle_hmatrix(torch_cuda, slab, name):
    mesh, built = slab
    A, H = built[name]
    rng = np.random.default_rng(17)
    x = (rng.normal(size=(2, A.n)) + 1j * rng.normal(size=(2, A.n))).astype(np.complex64)
    xt = torch_cuda.from_numpy(x).cuda()
    yt = torch_cuda.empty_like(xt)
    A.apply(xt, yt, n_levels=-1, fp64_accumulate=True)
    ref = H.from_tree(H.apply(H.to_tree(x.T.astype(np.complex128)))).T
    assert rel_err(yt.cpu().numpy(), ref) < 5 * TOL


@pytest.mark.parametrize("levels,refine", [(1, True), (1, False), (-1, False)])
def test_swg_series_solve_parity(torch_cuda, slab, levels, refine):
    # the oracle's own operator, imported: both sides run the same K-term series
    import synth
    from oracle import series
    mesh, built = slab
    _, H = built["binary_leaf16_c1"]
    A = gpu_operator(H)
    k, p = synth.random_incidences(16, seed=4)
    b = mesh.rhs(k, p)
    lv = H.n_levels if levels < 0 else levels
    ref = series.solve(H, b, K=2, levels=lv, nested_form=True, refine=refine).T
    bt = torch_cuda.from_numpy(b.T.astype(np.complex64).copy()).cuda()
    xt = torch_cuda.empty_like(bt)
    A.solve(bt, xt, n_terms=2, n_levels=levels, nested=True, refine=refine)
    assert rel_err(xt.cpu().numpy(), ref) < TOL


# ------------------------------------------------------------- full size ----

@pytest.fixture(scope="module")
def cube(torch_cuda):
    import synth
    from oracle.swg import SWGMesh
    from paper_2307_03968_gb300.hm import HMatrix
    xyz, tet = synth.cube_tets(15, 1.0)
    eps = synth.random_permittivity(len(tet), 2.0, 6.0, seed=4)
    A = HMatrix.build(xyz, tet, eps_r=eps, leaf_size=64, arity=2, adm=1.0, aca_tol=TOL, levels=-1)
    A.factor_leaf()
    return A, SWGMesh(xyz, tet, eps)


def test_swg_full_size_product_rows_sampled(torch_cuda, cube):
    A, mesh = cube
    N = A.n
    assert N == 41850
    rng = np.random.default_rng(5)
    x = (rng.normal(size=N) + 1j * rng.normal(size=N)).astype(np.complex64)
    xt = torch_cuda.from_numpy(x[None, :]).cuda()
    yt = torch_cuda.empty_like(xt)
    A.apply(xt, yt, n_levels=-1, fp64_accumulate=True)
    y = yt.cpu().numpy()[0]
    rows = np.sort(rng.choice(N, 10, replace=False)).astype(np.int32)
    Z = mesh.fill(rows, np.arange(N, dtype=np.int32))
    # half storage mirrors the upper triangle: rebuild the rows of the mirrored matrix
    perm = A.perm()
    pos = np.empty(N, np.int64)
    pos[perm] = np.arange(N)
    cols = np.arange(N, dtype=np.int32)
    for q, i in enumerate(rows):
        lower = pos[cols] < pos[i]
        if lower.any():
            Z[q, lower] = mesh.fill(cols[lower], np.array([i], np.int32))[:, 0]
    ref = Z @ x.astype(np.complex128)
    assert np.linalg.norm(y[rows] - ref) / np.linalg.norm(ref) < 1e-3


def test_swg_full_size_rhs_and_reciprocity(torch_cuda, cube):
    import synth
    A, mesh = cube
    N = A.n
    k, p = synth.random_incidences(16, seed=4)
    bt = torch_cuda.empty((16, N), dtype=torch_cuda.complex64, device="cuda")
    A.rhs_plane_wave(k, p, bt)
    ref = mesh.rhs(k, p).T
    assert np.abs(bt.cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()
    xt = torch_cuda.empty_like(bt)
    A.solve(bt, xt, n_terms=2, n_levels=1, nested=True, refine=True)
    x = xt.cpu().numpy().astype(np.complex128)
    b = bt.cpu().numpy().astype(np.complex128)
    assert np.all(np.isfinite(x))
    G = b @ x.T                                      # G[a, c] = b_a^T x_c
    gap = np.abs(G - G.T).max() / np.abs(G).max()
    assert gap < 1e-4, gap


def test_dielectric_ball_rcs_matches_oracle_and_mie(torch_cuda):
    # a homogeneous dielectric ball (eps_r = 2, radius 0.15 wavelength, 864 SWG unknowns) built on the GPU; the
    # series converges here (rho < 1), K = 16 terms: the bistatic RCS of the GPU solution is within 0.2 dB of the
    # oracle's series solution (the task's RCS bar) and within 0.3 dB of the Mie series of the equal-volume sphere
    import synth
    from oracle.swg import SWGMesh
    from oracle.hmatrix import HMatrix as OH
    from oracle import series, rcs, mie
    from paper_2307_03968_gb300.hm import HMatrix
    xyz, tet = synth.ball_tets(4, 0.15)
    eps = np.full(len(tet), 2.0)
    kw = dict(leaf_size=32, arity=2, adm=1.0, aca_tol=TOL)
    A = HMatrix.build(xyz, tet, eps_r=eps, levels=-1, **kw)
    A.factor_leaf()
    kh, ph = np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]])
    bt = torch_cuda.empty((1, A.n), dtype=torch_cuda.complex64, device="cuda")
    A.rhs_plane_wave(kh, ph, bt)
    xt = torch_cuda.empty_like(bt)
    A.solve(bt, xt, n_terms=16, n_levels=-1, nested=False)
    x = xt.cpu().numpy()[0].astype(np.complex128)
    m = SWGMesh(xyz, tet, eps)
    H = OH(m, **kw)
    xo = series.solve(H, m.rhs(kh, ph), K=16, levels=-1, nested_form=False)[:, 0]
    th = np.radians([0.0, 30.0, 60.0, 120.0, 150.0, 180.0])
    gpu = rcs.db(rcs.bistatic_theta_pol(m, x, th))
    orc = rcs.db(rcs.bistatic_theta_pol(m, xo, th))
    p = xyz[tet]
    vol = np.abs(np.einsum('ij,ij->i', np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])).sum() / 6
    a = (3 * vol / (4 * np.pi)) ** (1 / 3)
    ref = rcs.db(mie.dielectric_bistatic_eplane(a, 1.0, 2.0, th))
    assert np.abs(gpu - orc).max() < 0.2, gpu - orc
    assert np.abs(gpu - ref).max() < 0.3, gpu - ref
