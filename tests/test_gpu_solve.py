"""GPU parity of the power-series solve through the C ABI against the oracle.

Both sides solve the SAME operator: the oracle's complex128 H-Matrix is handed
to the library with hm_build_from_blocks (rounded to complex64 on the device,
self blocks kept in complex128 for the FP64 leaf factorisation).

Tolerance (stated per test): the complex64 path must reach max-column relative
error <= 1e-4 against the complex128 oracle for the same K, levels, form and
refinement; the FP64 path <= 1e-9.
"""

import numpy as np
import pytest

from hm_testutil import export_oracle, gpu_operator, rel_err

pytestmark = pytest.mark.gpu

TOL32 = 1e-4
TOL64 = 1e-9


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03968_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def cfg1(sphere_small):
    """PEC sphere 0.3 lambda, 1,920 RWG, octree leaf 32, 2-diameter admissibility."""
    from oracle.hmatrix import HMatrix
    return HMatrix(sphere_small, leaf_size=32, arity=8, adm=2.0, aca_tol=1e-4)


@pytest.fixture(scope="module")
def ml2(sphere_small):
    """Binary tree, leaf 32, eta = 1: near blocks plus far blocks on two levels."""
    from oracle.hmatrix import HMatrix
    return HMatrix(sphere_small, leaf_size=32, arity=2, adm=1.0, aca_tol=1e-4)


@pytest.fixture(scope="module")
def odd(sphere_small):
    """Binary tree, leaf 16: 128 leaves of 15 unknowns (odd, padded on the device),
    far blocks on several levels."""
    from oracle.hmatrix import HMatrix
    return HMatrix(sphere_small, leaf_size=16, arity=2, adm=1.0, aca_tol=1e-4)


def rhs(mesh, n, seed):
    from synth import random_incidences
    k, p = random_incidences(n, seed)
    return mesh.rhs(k, p)            # (N, n)


def gpu_solve(torch, A, b, dtype, **kw):
    bt = torch.from_numpy(np.ascontiguousarray(b.T)).to(dtype).cuda()
    xt = torch.empty_like(bt)
    A.solve(bt, xt, **kw)
    torch.cuda.synchronize()
    return xt.cpu().numpy()


@pytest.mark.parametrize("K", [0, 1, 2, 3])
def test_leaf_level_series_config1(torch_cuda, sphere_small, cfg1, K):
    from oracle import series
    b = rhs(sphere_small, 1, 21)
    ref = series.solve(cfg1, b, K=K, levels=1).T
    A = gpu_operator(cfg1)
    x = gpu_solve(torch_cuda, A, b, torch_cuda.complex64, n_terms=K, n_levels=1)
    assert rel_err(x, ref) < TOL32


@pytest.mark.parametrize("levels,nested,refine", [(1, True, False), (2, True, False), (2, False, False),
                                                  (2, True, True), (-1, False, True)])
def test_multilevel_forms(torch_cuda, sphere_small, ml2, levels, nested, refine):
    from oracle import series
    b = rhs(sphere_small, 3, 22)
    ref = series.solve(ml2, b, K=2, levels=levels, nested_form=nested, refine=refine).T
    A = gpu_operator(ml2)
    x = gpu_solve(torch_cuda, A, b, torch_cuda.complex64, n_terms=2, n_levels=levels, nested=nested,
                  refine=refine)
    assert rel_err(x, ref) < TOL32


def test_odd_leaves_many_levels(torch_cuda, sphere_small, odd):
    from oracle import series
    assert all(n % 2 == 1 for (_, n) in odd.leaves) and odd.n_levels >= 2
    b = rhs(sphere_small, 2, 23)
    for levels, nested in ((1, True), (-1, False), (odd.n_levels, True)):
        ref = series.solve(odd, b, K=2, levels=levels, nested_form=nested).T
        A = gpu_operator(odd)
        x = gpu_solve(torch_cuda, A, b, torch_cuda.complex64, n_terms=2, n_levels=levels, nested=nested)
        assert rel_err(x, ref) < TOL32, (levels, nested)


def test_fp64_path(torch_cuda, sphere_small, ml2):
    from oracle import series
    b = rhs(sphere_small, 2, 24)
    A = gpu_operator(ml2, keep_fp64=True)
    for levels, nested in ((1, True), (2, True), (2, False)):
        ref = series.solve(ml2, b, K=2, levels=levels, nested_form=nested).T
        x = gpu_solve(torch_cuda, A, b, torch_cuda.complex128, n_terms=2, n_levels=levels, nested=nested,
                      fp64=True)
        assert rel_err(x, ref) < TOL64, (levels, nested)


def test_apply_matches_oracle(torch_cuda, sphere_small, ml2):
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, ml2.N)) + 1j * rng.normal(size=(2, ml2.N))
    A = gpu_operator(ml2)
    x32 = x.astype(np.complex64)
    for levels in (1, 2):
        ref = ml2.from_tree(ml2.apply(ml2.to_tree(x32.T.astype(np.complex128)), levels)).T
        xt = torch_cuda.from_numpy(x32).cuda()
        for acc64, tol in ((True, 1e-6), (False, 1e-5)):
            yt = torch_cuda.empty_like(xt)
            A.apply(xt, yt, n_levels=levels, fp64_accumulate=acc64)
            assert rel_err(yt.cpu().numpy(), ref) < tol


def test_host_buffer_solve_equals_device_solve(torch_cuda, sphere_small, cfg1):
    from oracle import series
    b = rhs(sphere_small, 2, 25)
    A = gpu_operator(cfg1)
    xd = gpu_solve(torch_cuda, A, b, torch_cuda.complex64, n_terms=2, n_levels=1)
    xh = A.solve_host(b.T, n_terms=2, n_levels=1)
    assert rel_err(xh, xd) < 1e-6
    assert rel_err(xh, series.solve(cfg1, b, K=2, levels=1).T) < TOL32
    # page-locked buffers with leading dimension N go without the staging copies, with a
    # refined solve too; the result must be the same
    bp = torch_cuda.from_numpy(np.ascontiguousarray(b.T.astype(np.complex64))).pin_memory().numpy()
    xp = torch_cuda.empty(bp.shape, dtype=torch_cuda.complex64).pin_memory().numpy()
    xp[:] = np.nan
    out = A.solve_host(bp, n_terms=2, n_levels=1, out=xp)
    assert out is xp and rel_err(xp, xd) < 1e-6
    xr = A.solve_host(b.T, n_terms=2, n_levels=1, refine=True)
    xp[:] = np.nan
    A.solve_host(bp, n_terms=2, n_levels=1, refine=True, out=xp)
    assert rel_err(xp, xr) < 1e-6


def test_single_leaf_is_exact_solve(torch_cuda):
    from synth import box_surface
    from oracle.rwg import RWGMesh
    from oracle.hmatrix import HMatrix
    from oracle import series
    xyz, tri = box_surface((0.2, 0.2, 0.2), (2, 2, 2))
    mesh = RWGMesh(xyz, tri)
    H = HMatrix(mesh, leaf_size=mesh.ne, arity=8)
    assert H.depth == 0 and not H.near
    b = rhs(mesh, 1, 26)
    ref = series.solve(H, b, K=2, levels=-1).T
    A = gpu_operator(H)
    x = gpu_solve(torch_cuda, A, b, torch_cuda.complex64, n_terms=2, n_levels=-1)
    assert rel_err(x, ref) < TOL32


def test_state_and_singular_errors(torch_cuda, cfg1):
    from paper_2307_03968_gb300.hm import HMatrix, HmError, HM_ERR_STATE, HM_ERR_SINGULAR
    perm, leaf_off, D, near, far = export_oracle(cfg1)
    A = HMatrix.from_blocks(perm, leaf_off, D, near, far)
    b = torch_cuda.zeros(cfg1.N, dtype=torch_cuda.complex64, device="cuda")
    x = torch_cuda.empty_like(b)
    with pytest.raises(HmError) as e:
        A.solve(b, x)
    assert e.value.status == HM_ERR_STATE
    D2 = [d.copy() for d in D]
    D2[5][:] = 0.0
    A2 = HMatrix.from_blocks(perm, leaf_off, D2, near, far)
    with pytest.raises(HmError) as e:
        A2.factor_leaf()
    assert e.value.status == HM_ERR_SINGULAR and "5" in str(e.value)
    # nrhs = 0 is a no-op
    A.factor_leaf()
    A.solve(b[:0].reshape(0, cfg1.N), x[:0].reshape(0, cfg1.N))


def test_layout_round_trip(torch_cuda, odd):
    """The device keeps exactly the imported tree, leaves and blocks."""
    A = gpu_operator(odd)
    assert np.array_equal(A.perm(), odd.perm)
    assert np.array_equal(A.leaves(), [0] + [o + n for (o, n) in odd.leaves])
    r0, c0, m, n, k = A.blocks(1)
    assert np.sum(k == 0) == len(odd.near)
    B = A.block(1, 3)
    assert np.allclose(B, odd.near[3][4].astype(np.complex64), rtol=0, atol=0)
    lev = max(odd.far)
    r0, c0, m, n, k = A.blocks(lev)
    U, V = A.block(lev, 0)
    Uo, Vo = odd.far[lev][0][4], odd.far[lev][0][5]
    assert np.array_equal(U, Uo.astype(np.complex64)) and np.array_equal(V, Vo.astype(np.complex64))


def _rounded_operator(H):
    """The oracle's operator with every stored block rounded to complex64, as the
    library keeps it (complex128 copy so the oracle's products are FP64)."""
    import copy
    G = copy.copy(H)
    c64 = lambda a: a.astype(np.complex64).astype(np.complex128)
    G.D = [c64(d) for d in H.D]
    G.near = [(a, b, c, d, c64(B)) for (a, b, c, d, B) in H.near]
    G.far = {lev: [(a, b, c, d, c64(U), c64(V)) for (a, b, c, d, U, V) in lst] for lev, lst in H.far.items()}
    return G


@pytest.mark.parametrize("levels", [1, -1])
def test_residual_is_fp64_class(torch_cuda, ml2, levels):
    """b = A x rounded to complex64, so the true residual is ~1e-8 |A x|: an
    FP32-accumulated residual would be wrong by more than its own size; the
    FP64-class one must match the FP64 oracle residual to 1e-3 of |r|."""
    G = _rounded_operator(ml2)
    rng = np.random.default_rng(12)
    x = (rng.normal(size=(2, G.N)) + 1j * rng.normal(size=(2, G.N))).astype(np.complex64)
    y = np.ascontiguousarray(G.from_tree(G.apply(G.to_tree(x.T.astype(np.complex128)), levels)).T)  # FP64 A x
    b = np.ascontiguousarray(y.astype(np.complex64))
    r_ref = b.astype(np.complex128) - y
    A = gpu_operator(ml2)
    bt = torch_cuda.from_numpy(b).cuda()
    xt = torch_cuda.from_numpy(x).cuda()
    rt = torch_cuda.empty_like(bt)
    rr, bb = A.residual(bt, xt, rt, n_levels=levels)
    r = rt.cpu().numpy()
    assert rel_err(r, r_ref) < 1e-3
    assert np.allclose(rr, np.sum(np.abs(r_ref) ** 2, axis=1), rtol=1e-3)
    assert np.allclose(bb, np.sum(np.abs(b.astype(np.complex128)) ** 2, axis=1), rtol=1e-6)

