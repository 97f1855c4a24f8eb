"""The one-launch solve (hm_solve_opts.persistent): the whole solve as one
cooperative kernel whose CTAs walk the recorded steps with grid-wide barriers
in between.  It must give the oracle's result within the parity bar (1e-4,
max-column relative 2-norm, the same K, levels, form and refinement), agree
with the multi-kernel solve to FP32 rounding (1e-5), report divergence and
bounded-wait time-outs through the status word, and leave the handle usable.
Operators: the oracle's, handed over with hm_build_from_blocks (1,920-unknown
sphere: octree leaf 32 with the 2-diameter rule; binary tree leaf 32 with
eta = 1, far blocks on two levels; binary tree leaf 16, odd leaves of 15).
"""

import numpy as np
import pytest

from hm_testutil import gpu_operator, rel_err

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
def opers(sphere_small):
    from oracle.hmatrix import HMatrix
    return {"cfg1": HMatrix(sphere_small, leaf_size=32, arity=8, adm=2.0, aca_tol=1e-4),
            "ml2": HMatrix(sphere_small, leaf_size=32, arity=2, adm=1.0, aca_tol=1e-4),
            "odd": HMatrix(sphere_small, leaf_size=16, arity=2, adm=1.0, aca_tol=1e-4)}


def _rhs(mesh, n, seed):
    from synth import random_incidences
    return mesh.rhs(*random_incidences(n, seed))          # (N, n)


CASES = [("cfg1", 2, 1, True, True), ("cfg1", 0, 1, True, False), ("cfg1", 3, 1, True, True),
         ("ml2", 2, -1, True, True), ("ml2", 2, -1, False, True), ("ml2", 1, 2, True, False),
         ("odd", 2, -1, True, True), ("odd", 2, 1, False, False)]


@pytest.mark.parametrize("name,K,levels,nested,refine", CASES)
def test_one_launch_solve_matches_oracle(torch_cuda, sphere_small, opers, name, K, levels, nested, refine):
    from oracle import series
    H = opers[name]
    b = _rhs(sphere_small, 3, 41)
    ref = series.solve(H, b, K=K, levels=levels, nested_form=nested, refine=refine).T
    A = gpu_operator(H)
    bt = torch_cuda.from_numpy(np.ascontiguousarray(b.T.astype(np.complex64))).cuda()
    x_multi = torch_cuda.empty_like(bt)
    A.solve(bt, x_multi, n_terms=K, n_levels=levels, nested=nested, refine=refine)
    for graph in (False, True, True):               # eager, then graph capture and a replay
        xt = torch_cuda.full_like(bt, float("nan"))
        A.solve(bt, xt, n_terms=K, n_levels=levels, nested=nested, refine=refine, persistent=True, graph=graph)
        A.sync_status()
        x = xt.cpu().numpy()
        assert rel_err(x, ref) < 1e-4, graph
        assert rel_err(x, x_multi.cpu().numpy()) < 1e-5, graph


def test_one_launch_info_and_launch_count(torch_cuda, sphere_small, opers):
    H = opers["ml2"]
    b = _rhs(sphere_small, 2, 42)
    A = gpu_operator(H)
    bt = torch_cuda.from_numpy(np.ascontiguousarray(b.T.astype(np.complex64))).cuda()
    x1, x2 = torch_cuda.empty_like(bt), torch_cuda.empty_like(bt)
    s1 = A.solve(bt, x1, n_terms=2, n_levels=-1, refine=True, info=True)
    s2 = A.solve(bt, x2, n_terms=2, n_levels=-1, refine=True, info=True, persistent=True)
    assert s1.kernel_launches > 10 and s2.kernel_launches == 1
    assert s2.rel_residual == pytest.approx(s1.rel_residual, rel=1e-4)
    assert s2.bytes_streamed == s1.bytes_streamed


def test_one_launch_reports_divergence(torch_cuda, sphere_small, opers):
    from paper_2307_03968_gb300.hm import HmError, HM_ERR_DIVERGED
    H = opers["cfg1"]
    b = _rhs(sphere_small, 2, 43).T.astype(np.complex64)
    bad = b.copy()
    bad[1, 5] = np.inf
    A = gpu_operator(H)
    bt = torch_cuda.from_numpy(np.ascontiguousarray(bad)).cuda()
    xt = torch_cuda.empty_like(bt)
    A.solve(bt, xt, n_terms=2, n_levels=1, refine=True, persistent=True)
    with pytest.raises(HmError) as e:
        A.sync_status()
    assert e.value.status == HM_ERR_DIVERGED


def test_one_launch_barrier_timeout_is_reported_and_recovers(torch_cuda, sphere_small, opers):
    # with a wait limit of zero polls every CTA but the last to arrive gives up at the first
    # grid barrier and leaves; the last one gives up at the next barrier: HM_ERR_TIMEOUT
    from oracle import series
    from paper_2307_03968_gb300.hm import HmError, HM_ERR_TIMEOUT
    H = opers["cfg1"]
    b = _rhs(sphere_small, 1, 44)
    A = gpu_operator(H)
    bt = torch_cuda.from_numpy(np.ascontiguousarray(b.T.astype(np.complex64))).cuda()
    xt = torch_cuda.empty_like(bt)
    A.set_wait_limit(0)
    A.solve(bt, xt, n_terms=2, n_levels=1, refine=True, persistent=True, graph=False)
    with pytest.raises(HmError) as e:
        A.sync_status()
    assert e.value.status == HM_ERR_TIMEOUT
    A.set_wait_limit(-1)
    A.solve(bt, xt, n_terms=2, n_levels=1, refine=True, persistent=True)
    A.sync_status()
    ref = series.solve(H, b, K=2, levels=1, refine=True).T
    assert rel_err(xt.cpu().numpy(), ref) < 1e-4
