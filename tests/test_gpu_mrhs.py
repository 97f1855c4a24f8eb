"""Many right-hand sides: the block product that reads each block once per
chunk of right-hand sides (shared-memory staged, k_mrhs.cu) against the same
product taken one right-hand side at a time (the single-RHS kernel), on the
same operator, in FP32 arithmetic.  Both accumulate with atomics in an
unspecified order, so they agree to FP32 rounding: relative 2-norm per column
<= 1e-5.  RHS counts cover every chunk width (8, 16, 32), ragged last chunks,
and the switch-over point; the operators mix dense blocks, low-rank blocks
that fit shared memory, and blocks that do not (leaves of 108 unknowns)."""

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


@pytest.fixture(scope="module")
def operators(torch_cuda):
    import synth
    from paper_2307_03968_gb300.hm import HMatrix
    ops = {}
    xyz, tri = synth.icosphere(3, 0.3)
    ops["rwg_binary15"] = HMatrix.build(xyz, tri, leaf_size=15, arity=2, adm=1.0, aca_tol=1e-4, levels=-1)
    xyz, tet = synth.cube_tets(4, 1.0)
    xyz = xyz * np.array([2.0, 0.25, 0.125])
    eps = synth.random_permittivity(len(tet), 2.0, 6.0, seed=4)
    ops["swg_slab"] = HMatrix.build(xyz, tet, eps_r=eps, leaf_size=16, arity=2, adm=1.0, aca_tol=1e-4, levels=-1)
    # 864 unknowns halved three times: leaves of 108, dense blocks too large for shared memory
    ops["swg_slab_leaf112"] = HMatrix.build(xyz, tet, eps_r=eps, leaf_size=112, arity=2, adm=1.0, aca_tol=1e-6,
                                            levels=-1)
    # octree leaves of up to 64 unknowns: tensor-core products at full operand width (N = 128)
    xyz, tri = synth.icosphere(3, 0.3)
    ops["rwg_octree64"] = HMatrix.build(xyz, tri, leaf_size=64, arity=8, adm=2.0, aca_tol=1e-4, levels=-1)
    for A in ops.values():
        A.factor_leaf()
    return ops


PRODUCT_KERNELS = [0, 8, 16, 32, 1016]   # one RHS at a time, SIMT chunks, tensor-core dense blocks


@pytest.mark.parametrize("name", ["rwg_binary15", "swg_slab", "swg_slab_leaf112", "rwg_octree64"])
@pytest.mark.parametrize("nrhs", [3, 4, 7, 8, 13, 16, 33, 70])
def test_many_rhs_product_equals_column_products(torch_cuda, operators, name, nrhs):
    A = operators[name]
    N = A.n
    rng = np.random.default_rng(nrhs)
    x = (rng.normal(size=(nrhs, N)) + 1j * rng.normal(size=(nrhs, N))).astype(np.complex64)
    xt = torch_cuda.from_numpy(x).cuda()
    ref = np.empty_like(x)
    for r in range(nrhs):
        y1 = torch_cuda.empty((1, N), dtype=torch_cuda.complex64, device="cuda")
        A.apply(xt[r:r + 1].contiguous(), y1, n_levels=-1, fp64_accumulate=False)
        ref[r] = y1.cpu().numpy()[0]
    kernels = PRODUCT_KERNELS if nrhs >= 4 else [None]
    for kern in kernels:
        if kern is not None:
            A.set_tuning(nrhs, kern, 0)
        yt = torch_cuda.empty_like(xt)
        A.apply(xt, yt, n_levels=-1, fp64_accumulate=False)
        got = yt.cpu().numpy()
        for r in range(nrhs):
            err = np.linalg.norm(got[r] - ref[r]) / np.linalg.norm(ref[r])
            assert err < 1e-5, (kern, r, err)


@pytest.mark.parametrize("name", ["rwg_binary15", "swg_slab", "rwg_octree64"])
@pytest.mark.parametrize("nrhs", [128, 130, 261])
def test_tensor_core_product_over_several_tiles(torch_cuda, operators, name, nrhs):
    # tiles of 128 right-hand sides (full, ragged, three tiles) on the tensor cores
    # against one right-hand side at a time, FP32 rounding apart (3xTF32 products)
    A = operators[name]
    N = A.n
    rng = np.random.default_rng(nrhs + 5)
    x = (rng.normal(size=(nrhs, N)) + 1j * rng.normal(size=(nrhs, N))).astype(np.complex64)
    xt = torch_cuda.from_numpy(x).cuda()
    ref = torch_cuda.empty_like(xt)
    A.set_tuning(nrhs, 0, 0)
    A.apply(xt, ref, n_levels=-1, fp64_accumulate=False)
    A.set_tuning(nrhs, 1016, 0)
    yt = torch_cuda.empty_like(xt)
    A.apply(xt, yt, n_levels=-1, fp64_accumulate=False)
    got, want = yt.cpu().numpy(), ref.cpu().numpy()
    err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
    assert err.max() < 1e-5, err.max()


def test_operators_exercise_both_kernels(operators):
    big = 0
    small = 0
    for A in operators.values():
        for lev in range(1, A.info().n_levels + 1):
            r0, c0, m, n, k = A.blocks(lev)
            fits = (m <= 64) & (n <= 64) & (k <= 32)
            small += int(fits.sum())
            big += int((~fits).sum())
    assert small > 100 and big > 10


@pytest.mark.parametrize("name", ["rwg_binary15", "swg_slab", "swg_slab_leaf112"])
@pytest.mark.parametrize("nrhs", [4, 9, 16, 21])
def test_many_rhs_residual_equals_column_residuals(torch_cuda, operators, name, nrhs):
    # FP64-class residual r = b - A x: the multi-RHS kernel (chunks of up to 16,
    # blocks staged once) against one right-hand side at a time; both sum each
    # block in compensated FP32 and the blocks in FP64, in different orders
    A = operators[name]
    N = A.n
    rng = np.random.default_rng(100 + nrhs)
    x = (rng.normal(size=(nrhs, N)) + 1j * rng.normal(size=(nrhs, N))).astype(np.complex64)
    xt = torch_cuda.from_numpy(x).cuda()
    ax = torch_cuda.empty_like(xt)
    A.apply(xt, ax, n_levels=-1, fp64_accumulate=True)
    # b close to A x, so that the residual is small and its FP64-class accuracy matters
    b = ax.cpu().numpy() + (1e-5 * (rng.normal(size=(nrhs, N)) + 1j * rng.normal(size=(nrhs, N)))).astype(np.complex64)
    bt = torch_cuda.from_numpy(b).cuda()
    rt = torch_cuda.empty_like(xt)
    rr, bb = A.residual(bt, xt, rt, n_levels=-1)
    got = rt.cpu().numpy()
    for r in range(nrhs):
        r1 = torch_cuda.empty((1, N), dtype=torch_cuda.complex64, device="cuda")
        rr1, bb1 = A.residual(bt[r:r + 1].contiguous(), xt[r:r + 1].contiguous(), r1, n_levels=-1)
        ref = r1.cpu().numpy()[0]
        assert np.abs(got[r] - ref).max() <= 1e-6 * np.abs(ref).max(), r
        assert rr[r] == pytest.approx(rr1[0], rel=1e-9)
        assert bb[r] == pytest.approx(bb1[0], rel=1e-12)


def test_autotuner_records_a_choice(torch_cuda, operators):
    from paper_2307_03968_gb300.hm import HmError, HM_ERR_STATE
    A = operators["swg_slab"]
    N = A.n
    rng = np.random.default_rng(7)
    x = (rng.normal(size=(24, N)) + 1j * rng.normal(size=(24, N))).astype(np.complex64)
    xt = torch_cuda.from_numpy(x).cuda()
    yt = torch_cuda.empty_like(xt)
    A.apply(xt, yt, n_levels=-1, fp64_accumulate=False)      # first call with 24 RHS: tunes
    prod_rb, res_rb, prod_ms, res_ms = A.tuning(24)
    assert prod_rb in (0, 8, 16, 32) and res_rb in (0, 8, 16, 1017)
    assert prod_ms > 0 and res_ms > 0
    again = torch_cuda.empty_like(xt)
    A.apply(xt, again, n_levels=-1, fp64_accumulate=False)   # tuned choice is kept
    assert A.tuning(24) == (prod_rb, res_rb, prod_ms, res_ms)
    assert np.allclose(again.cpu().numpy(), yt.cpu().numpy(), rtol=1e-5, atol=1e-6 * np.abs(yt.cpu().numpy()).max())
    with pytest.raises(HmError) as e:
        A.tuning(3)                                           # below the many-RHS threshold: nothing to tune
    assert e.value.status == HM_ERR_STATE


@pytest.mark.parametrize("name", ["rwg_binary15", "swg_slab", "rwg_octree64"])
@pytest.mark.parametrize("nrhs", [4, 17, 40])
def test_owner_residual_equals_partial_slot_residual(torch_cuda, operators, name, nrhs):
    # the owner-computes FP64-class residual (one CTA per output cluster and 16 RHS,
    # FP64 sums without partial slots) against the partial-slot kernel (one RHS at a
    # time) on the leaf level, where every block is small; both are FP64-class, so
    # they agree far below the complex64 rounding of r
    A = operators[name]
    N = A.n
    rng = np.random.default_rng(200 + nrhs)
    x = (rng.normal(size=(nrhs, N)) + 1j * rng.normal(size=(nrhs, N))).astype(np.complex64)
    xt = torch_cuda.from_numpy(x).cuda()
    ax = torch_cuda.empty_like(xt)
    A.apply(xt, ax, n_levels=1, fp64_accumulate=True)
    b = ax.cpu().numpy() + (1e-5 * (rng.normal(size=(nrhs, N)) + 1j * rng.normal(size=(nrhs, N)))).astype(np.complex64)
    bt = torch_cuda.from_numpy(b).cuda()
    A.set_tuning(nrhs, 0, 0)
    r0 = torch_cuda.empty_like(xt)
    rr0, bb0 = A.residual(bt, xt, r0, n_levels=1)
    A.set_tuning(nrhs, 0, 1017)
    r1 = torch_cuda.empty_like(xt)
    rr1, bb1 = A.residual(bt, xt, r1, n_levels=1)
    want, got = r0.cpu().numpy(), r1.cpu().numpy()
    for r in range(nrhs):
        assert np.abs(got[r] - want[r]).max() <= 1e-6 * np.abs(want[r]).max(), r
        assert rr1[r] == pytest.approx(rr0[r], rel=1e-9)
        assert bb1[r] == pytest.approx(bb0[r], rel=1e-12)
    # a refined solve through the owner residual equals the one through the partial slots
    A.set_tuning(nrhs, 0, 0)
    s0 = torch_cuda.empty_like(xt)
    A.solve(bt, s0, n_terms=2, n_levels=1, refine=True)
    A.set_tuning(nrhs, 0, 1017)
    s1 = torch_cuda.empty_like(xt)
    A.solve(bt, s1, n_terms=2, n_levels=1, refine=True)
    a0, a1 = s0.cpu().numpy(), s1.cpu().numpy()
    assert (np.linalg.norm(a1 - a0, axis=1) / np.linalg.norm(a0, axis=1)).max() < 1e-6
