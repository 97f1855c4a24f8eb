"""The library's convergence report (hm_estimate_norms, hm_info, hm_solve_info)
against the oracle's dense level operators.

Paper §IV eqs. 20-22: the solve truncates the power series of (I + U)^{-1},
U_l = D^{-1} M_l; §V states its operating bound as a norm of U below 0.1.  The
series converges as K grows exactly when the spectral radius of U_l is below
one.  The oracle forms U_l densely (D^{-1} applied by LU solves to every column
of M_l) and takes its largest singular value and the largest modulus of its
eigenvalues with LAPACK; the GPU estimates both by power iterations (the norm
as a lower bound that rises to it).  Tolerances: 64 steps land within 1 % of
both on these operators in a float64 emulation of the same iterations; the test
allows 3 %.  The default of hm_factor_leaf (32 steps) is allowed 3 % on the
norm and 6 % on the spectral radius.
"""

import numpy as np
import pytest

import synth
from hm_testutil import gpu_operator

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03968_gb300 import build
    build.build()
    return torch


def dense_level_stats(H):
    """(sigma_max, rho) of U_l = D^{-1} M_l per level l = 1..n_levels (None if empty)."""
    out = []
    eye = np.eye(H.N, dtype=np.complex128)
    for lev in range(1, H.n_levels + 1):
        M = H.apply_M(lev, eye)
        if not np.any(M):
            out.append(None)
            continue
        U = H.solve_D(M)
        out.append((np.linalg.svd(U, compute_uv=False)[0], np.abs(np.linalg.eigvals(U)).max()))
    return out


def check(A, stats, norm_tol, rho_tol):
    norm, rho = A.norm_estimates()
    for lev, st in enumerate(stats, start=1):
        if st is None:
            assert norm[lev - 1] == 0.0 and rho[lev - 1] == 0.0
            continue
        sigma, r = st
        assert sigma * (1 - norm_tol) <= norm[lev - 1] <= sigma * (1 + 1e-4), (lev, norm[lev - 1], sigma)
        assert abs(rho[lev - 1] - r) <= rho_tol * r, (lev, rho[lev - 1], r)


def test_sphere_leaf_level_diverges(torch_cuda, sphere_small):
    # 1,920 RWG unknowns, octree leaf 32, 2-diameter rule: only the leaf level; rho(U_1) = 2.57
    from oracle.hmatrix import HMatrix as OracleH
    H = OracleH(sphere_small, leaf_size=32, arity=8, adm=2.0, aca_tol=1e-4)
    stats = dense_level_stats(H)
    A = gpu_operator(H)
    assert A.info().norm_iters == 32
    check(A, stats, 0.03, 0.06)                      # the estimate hm_factor_leaf made
    A.estimate_norms(64)
    assert A.info().norm_iters == 64
    check(A, stats, 0.03, 0.03)
    assert stats[0][1] > 2.0                         # the S-EFIE sphere: the series diverges
    b = torch_cuda.from_numpy(synth_rhs(sphere_small, H.N)).cuda()
    x = torch_cuda.empty_like(b)
    si = A.solve(b, x, n_terms=2, n_levels=1, refine=True, info=True)
    assert si.convergent == 0
    assert si.rho_est[0] == pytest.approx(A.norm_estimates()[1][0])
    assert si.rel_residual > 0.0


def test_multilevel_operator(torch_cuda, sphere_small):
    # binary tree, eq. 7 with eta = 1: far blocks on two levels (rho(U_2) = 0.085, below 0.1)
    from oracle.hmatrix import HMatrix as OracleH
    H = OracleH(sphere_small, leaf_size=32, arity=2, adm=1.0, aca_tol=1e-4)
    stats = dense_level_stats(H)
    assert len(stats) >= 2
    A = gpu_operator(H)
    A.estimate_norms(64)
    check(A, stats, 0.03, 0.03)


def test_dielectric_slab_converges(torch_cuda):
    # the paper's dielectric setting (eps_r = 2, binary tree, eta = 1, ACA 1e-3): rho(U_1) = 0.65 < 1
    from oracle.hmatrix import HMatrix as OracleH
    from oracle.swg import SWGMesh
    xyz, tet = synth.box_tets((2.0, 0.5, 0.1), (20, 5, 1))
    mesh = SWGMesh(xyz, tet, 2.0)
    H = OracleH(mesh, leaf_size=32, arity=2, adm=1.0, aca_tol=1e-3)
    stats = dense_level_stats(H)
    A = gpu_operator(H)
    A.estimate_norms(64)
    check(A, stats, 0.03, 0.03)
    b = torch_cuda.from_numpy(synth_rhs(mesh, H.N)).cuda()
    x = torch_cuda.empty_like(b)
    si = A.solve(b, x, n_terms=2, n_levels=-1, refine=False, info=True)
    assert si.convergent == 1
    assert all(si.rho_est[i] < 1.0 for i in range(si.levels_used))


def test_estimate_arguments(torch_cuda, sphere_tiny):
    from oracle.hmatrix import HMatrix as OracleH
    from paper_2307_03968_gb300 import hm
    H = OracleH(sphere_tiny, leaf_size=32, arity=2, adm=1.0, aca_tol=1e-4)
    A = gpu_operator(H)
    L = hm.load()
    assert L.hm_estimate_norms(A._h, 1, hm._stream(None)) == hm.HM_ERR_ARG
    assert L.hm_estimate_norms(A._h, 5000, hm._stream(None)) == hm.HM_ERR_ARG


def synth_rhs(mesh, n):
    k, p = synth.plane_wave_z()
    return mesh.rhs(k, p)[:, 0].astype(np.complex64).reshape(1, n)
