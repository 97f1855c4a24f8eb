"""Every many-right-hand-side kernel choice, pinned with hm_set_tuning, against
the oracle directly (not against another CUDA kernel).

Choices (include/hmps.h, hm_set_tuning): product 0 (one right-hand side at a
time), 8 / 16 / 32 (shared-memory SIMT chunks), 1016 (tcgen05 3xTF32 tensor-core
products of the blocks of at most 64 x 64, rank <= 32); residual 0, 8, 16
(partial-slot FP64-class products) and 1017 (owner-computes FP64-class
products, where every level of the call holds only such blocks, else the
one-at-a-time partial-slot kernel).

Operators (the oracle's, handed over with hm_build_from_blocks):
  - binary tree, leaf 32, eta = 1 on the 1,920-unknown sphere: leaves of 30, far
    blocks on two levels, every block small (the owner residual applies to all
    levels);
  - binary tree, leaf 64, eta = 1 on the same sphere: leaves of 60 (full
    128-column tensor-core operands, as in the 30,720-unknown workload), coarse
    far blocks larger than 64 x 64 that every choice hands to the one-at-a-time
    kernel.

Bars (the parity bars of the other tests): a refined K = 2 solve on 130
right-hand sides (two tensor-core tiles of 128, the second ragged) within 1e-4
of series.solve column by column; hm_apply within 1e-5 of the oracle's FP64
product; the FP64-class residual of 20 right-hand sides (one full and one
ragged group of 16) within 1e-3 of |r| of the FP64 oracle residual, on a
right-hand side b = fl32(A x) whose true residual is ~1e-8 |A x|.
"""

import numpy as np
import pytest

from hm_testutil import gpu_operator, rel_err

pytestmark = pytest.mark.gpu

COMBOS = [(0, 0), (8, 8), (16, 16), (32, 0), (1016, 1017)]   # every product and every residual choice


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03968_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def opers(sphere_small):
    from oracle.hmatrix import HMatrix
    return {"leaf32": HMatrix(sphere_small, leaf_size=32, arity=2, adm=1.0, aca_tol=1e-4),
            "leaf64": HMatrix(sphere_small, leaf_size=64, arity=2, adm=1.0, aca_tol=1e-4)}


def _rounded(H):
    """The oracle's operator with every stored block rounded to complex64, as the
    library keeps it (complex128 arithmetic on the rounded values)."""
    import copy
    G = copy.copy(H)
    c64 = lambda a: a.astype(np.complex64).astype(np.complex128)
    G.D = [c64(d) for d in H.D]
    G.near = [(a, b, c, d, c64(B)) for (a, b, c, d, B) in H.near]
    G.far = {lev: [(a, b, c, d, c64(U), c64(V)) for (a, b, c, d, U, V) in lst] for lev, lst in H.far.items()}
    return G


@pytest.mark.parametrize("name", ["leaf32", "leaf64"])
@pytest.mark.parametrize("levels", [1, -1])
def test_refined_solve_every_choice(torch_cuda, sphere_small, opers, name, levels):
    from synth import random_incidences
    from oracle import series
    H = opers[name]
    nr = 130
    k, p = random_incidences(nr, 131)
    b = sphere_small.rhs(k, p)                                   # (N, 130)
    ref = series.solve(H, b, K=2, levels=levels, refine=True).T
    A = gpu_operator(H)
    bt = torch_cuda.from_numpy(np.ascontiguousarray(b.T.astype(np.complex64))).cuda()
    for prod, res in COMBOS:
        A.set_tuning(nr, prod, res)
        xt = torch_cuda.full_like(bt, float("nan"))
        A.solve(bt, xt, n_terms=2, n_levels=levels, refine=True)
        A.sync_status()
        assert A.tuning(nr)[:2] == (prod, res)
        x = xt.cpu().numpy()
        errs = [np.linalg.norm(x[j] - ref[j]) / np.linalg.norm(ref[j]) for j in range(nr)]
        assert max(errs) < 1e-4, (prod, res, max(errs), int(np.argmax(errs)))


@pytest.mark.parametrize("name", ["leaf32", "leaf64"])
@pytest.mark.parametrize("levels", [1, -1])
def test_product_every_choice(torch_cuda, opers, name, levels):
    H = opers[name]
    nr = 130
    rng = np.random.default_rng(132)
    x = (rng.normal(size=(nr, H.N)) + 1j * rng.normal(size=(nr, H.N))).astype(np.complex64)
    ref = H.from_tree(H.apply(H.to_tree(x.T.astype(np.complex128)), levels)).T
    A = gpu_operator(H)
    xt = torch_cuda.from_numpy(x).cuda()
    for prod in (0, 8, 16, 32, 1016):
        A.set_tuning(nr, prod, 0)
        yt = torch_cuda.full_like(xt, float("nan"))
        A.apply(xt, yt, n_levels=levels, fp64_accumulate=False)
        A.sync_status()
        y = yt.cpu().numpy()
        errs = [np.linalg.norm(y[j] - ref[j]) / np.linalg.norm(ref[j]) for j in range(nr)]
        assert max(errs) < 1e-5, (prod, max(errs))


@pytest.mark.parametrize("name", ["leaf32", "leaf64"])
@pytest.mark.parametrize("levels", [1, -1])
def test_fp64_class_residual_every_choice(torch_cuda, opers, name, levels):
    H = opers[name]
    G = _rounded(H)
    nr = 20
    rng = np.random.default_rng(133)
    x = (rng.normal(size=(nr, G.N)) + 1j * rng.normal(size=(nr, G.N))).astype(np.complex64)
    y = np.ascontiguousarray(G.from_tree(G.apply(G.to_tree(x.T.astype(np.complex128)), levels)).T)   # FP64 A x
    b = np.ascontiguousarray(y.astype(np.complex64))
    r_ref = b.astype(np.complex128) - y                          # ~1e-8 |A x|
    A = gpu_operator(H)
    bt = torch_cuda.from_numpy(b).cuda()
    xt = torch_cuda.from_numpy(x).cuda()
    for res in (0, 8, 16, 1017):
        A.set_tuning(nr, 0, res)
        rt = torch_cuda.full_like(bt, float("nan"))
        rr, bb = A.residual(bt, xt, rt, n_levels=levels)
        r = rt.cpu().numpy()
        assert rel_err(r, r_ref) < 1e-3, res
        assert np.allclose(rr, np.sum(np.abs(r_ref) ** 2, axis=1), rtol=1e-3), res
        assert np.allclose(bb, np.sum(np.abs(b.astype(np.complex128)) ** 2, axis=1), rtol=1e-6), res
    # the product with FP64-class accumulation (hm_apply, fp64_accumulate) takes the residual kernels too
    for res in (0, 8, 16, 1017):
        A.set_tuning(nr, 0, res)
        yt = torch_cuda.full_like(xt, float("nan"))
        A.apply(xt, yt, n_levels=levels, fp64_accumulate=True)
        assert rel_err(yt.cpu().numpy(), y) < 1e-6, res


def _abs_operator(G):
    """The operator with every stored factor replaced by its elementwise modulus: applied to
    |x| it gives, per row, the sum of the moduli of the terms the residual sums (for a
    low-rank block, sum_l |U_il| |V_lj| |x_j|), the scale of error-free summation."""
    import copy
    Q = copy.copy(G)
    Q.D = [np.abs(d) for d in G.D]
    Q.near = [(a, b, c, d, np.abs(B)) for (a, b, c, d, B) in G.near]
    Q.far = {lev: [(a, b, c, d, np.abs(U), np.abs(V)) for (a, b, c, d, U, V) in lst] for lev, lst in G.far.items()}
    return Q


@pytest.mark.parametrize("name", ["leaf32", "leaf64"])
@pytest.mark.parametrize("levels", [1, -1])
def test_fp64_class_residual_special_cases(torch_cuda, opers, name, levels):
    """Cases with exact answers, through every residual choice.  x = 0: every grid
    is zero and r = b bit for bit.  b = 0, x = c_q e_{j_q} (one scaled unit vector
    per right-hand side): r = -c_q A e_{j_q}, a column of the operator.  Each entry
    must be within the complex64 rounding of r (2^-23 |r_i|) plus an FP64-class share
    of the sum of the moduli of its terms (s_i = sum_l |U_il| |V_lj| |c| for a low-rank
    block): a dropped term, a wrong sign or a transposed block is off by O(s_i)."""
    H = opers[name]
    G = _rounded(H)
    nr = 20
    rng = np.random.default_rng(134)
    A = gpu_operator(H)
    b = (rng.normal(size=(nr, H.N)) + 1j * rng.normal(size=(nr, H.N))).astype(np.complex64)
    bt = torch_cuda.from_numpy(b).cuda()
    x0 = torch_cuda.zeros_like(bt)
    js = rng.choice(H.N, nr, replace=False)
    c = (rng.normal(size=nr) + 1j * rng.normal(size=nr)).astype(np.complex64)
    X = np.zeros((nr, H.N), dtype=np.complex64)
    X[np.arange(nr), js] = c
    apply = lambda Q, v: np.ascontiguousarray(Q.from_tree(Q.apply(Q.to_tree(v.T.astype(np.complex128)), levels)).T)
    ref = -apply(G, X)
    scale = np.abs(apply(_abs_operator(G), np.abs(X))).real
    xt = torch_cuda.from_numpy(X).cuda()
    zt = torch_cuda.zeros_like(bt)
    for res in (0, 8, 16, 1017):
        A.set_tuning(nr, 0, res)
        rt = torch_cuda.full_like(bt, float("nan"))
        A.residual(bt, x0, rt, n_levels=levels)
        assert np.array_equal(rt.cpu().numpy(), b), res
        rt = torch_cuda.full_like(bt, float("nan"))
        A.residual(zt, xt, rt, n_levels=levels)
        r = rt.cpu().numpy().astype(np.complex128)
        assert np.all(np.isfinite(r)), res
        has = scale > 0
        assert np.all(r[~has] == 0), res                     # entries without terms are exactly zero
        excess = np.maximum(np.abs(r - ref) - 2.0 ** -23 * np.abs(ref), 0.0)[has] / scale[has]
        print("residual choice %d: worst error beyond the output rounding, in units of sum|terms|: %.2e"
              % (res, float(excess.max())))
        assert float(excess.max()) < 2.0 ** -30, res
