"""Failure paths, in the forms that leave the GPU usable: every device wait is
bounded and reports through the status word, bad data is reported, and an
oversize request is refused on the host.

- The tensor-core product's pipeline waits (mbarrier hand-offs between its
  copy, conversion and MMA roles) take their poll limit from hm_set_wait_limit.
  With a limit of zero every wait gives up at once: the kernel must record
  HM_ERR_TIMEOUT (read by hm_sync_status), drain its own copies and MMAs, free
  its tensor memory and return; the next product at the default limit must be
  correct (against the oracle's H-Matrix product).
- A non-finite right-hand side gives a non-finite solution, which the solve
  reports as HM_ERR_DIVERGED (through hm_sync_status, or directly when the call
  synchronises); the handle stays usable.
- A serving request that needs more device memory than the server's HBM budget
  is refused by hm_server_submit with HM_ERR_OOM; requests around it are served
  and equal the same requests solved alone.
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


def test_tensor_core_wait_timeout_is_reported_and_recovers(torch_cuda, sphere_small):
    from oracle.hmatrix import HMatrix as OracleH
    from paper_2307_03968_gb300.hm import HmError, HM_ERR_TIMEOUT
    H = OracleH(sphere_small, leaf_size=32, arity=8, adm=2.0, aca_tol=1e-4)
    A = gpu_operator(H)
    nr = 64
    rng = np.random.default_rng(91)
    x = (rng.normal(size=(nr, H.N)) + 1j * rng.normal(size=(nr, H.N))).astype(np.complex64)
    xt = torch_cuda.from_numpy(x).cuda()
    yt = torch_cuda.empty_like(xt)
    A.set_tuning(nr, 1016, 0)                       # the tensor-core product
    A.set_wait_limit(0)
    A.apply(xt, yt, n_levels=1, fp64_accumulate=False)
    with pytest.raises(HmError) as e:
        A.sync_status()
    assert e.value.status == HM_ERR_TIMEOUT
    A.sync_status()                                 # the status word was cleared by the read
    A.set_wait_limit(-1)
    A.apply(xt, yt, n_levels=1, fp64_accumulate=False)
    A.sync_status()
    ref = H.from_tree(H.apply(H.to_tree(x.T.astype(np.complex128)), 1)).T
    assert rel_err(yt.cpu().numpy(), ref) < 1e-5


def test_nonfinite_rhs_reports_diverged(torch_cuda, sphere_tiny):
    from oracle.hmatrix import HMatrix as OracleH
    from oracle import series
    from paper_2307_03968_gb300.hm import HmError, HM_ERR_DIVERGED
    H = OracleH(sphere_tiny, leaf_size=32, arity=2, adm=1.0, aca_tol=1e-4)
    A = gpu_operator(H)
    rng = np.random.default_rng(92)
    b = (rng.normal(size=(3, H.N)) + 1j * rng.normal(size=(3, H.N))).astype(np.complex64)
    bad = b.copy()
    bad[1, 17] = np.nan
    bt = torch_cuda.from_numpy(bad).cuda()
    xt = torch_cuda.empty_like(bt)
    A.solve(bt, xt, n_terms=2, n_levels=1, refine=True, graph=False)
    with pytest.raises(HmError) as e:
        A.sync_status()
    assert e.value.status == HM_ERR_DIVERGED
    with pytest.raises(HmError) as e:                # a synchronising call returns it directly
        A.solve(bt, xt, n_terms=2, n_levels=1, refine=True, info=True)
    assert e.value.status == HM_ERR_DIVERGED
    good = torch_cuda.from_numpy(b).cuda()           # the handle stays usable
    A.solve(good, xt, n_terms=2, n_levels=1, refine=True)
    A.sync_status()
    ref = series.solve(H, b.T.astype(np.complex128), K=2, levels=1, refine=True).T
    assert rel_err(xt.cpu().numpy(), ref) < 1e-4


def test_server_refuses_oversize_request(torch_cuda):
    from synth import icosphere
    from paper_2307_03968_gb300.hm import HMatrix, Server, HmError, HM_ERR_OOM
    xyz, tri = icosphere(2, 0.15)                    # 480 unknowns
    opts = dict(leaf_size=32, arity=8, adm=2.0, aca_tol=1e-4)
    sopts = dict(n_terms=2, n_levels=1, refine=True)
    A = HMatrix.build(xyz, tri, **opts)
    A.factor_leaf()
    # 2 MiB: a 64-column request alone needs 8 * 480 * 18 * 64 = 4.4 MB, a 2-column one 0.14 MB
    srv = Server(n_slots=2, hbm_budget_bytes=2 << 20, max_batch_rhs=64)
    op, n = srv.add_mesh(xyz, tri, **opts, **sopts)
    rng = np.random.default_rng(93)
    small = [(rng.normal(size=(2, n)) + 1j * rng.normal(size=(2, n))).astype(np.complex64) for _ in range(4)]
    reqs = [srv.submit(op, small[0]), srv.submit(op, small[1])]
    with pytest.raises(HmError) as e:
        srv.submit(op, np.zeros((64, n), np.complex64))
    assert e.value.status == HM_ERR_OOM
    reqs += [srv.submit(op, small[2]), srv.submit(op, small[3])]
    for b, r in zip(small, reqs):
        x, _ = srv.wait(r)
        bt = torch_cuda.from_numpy(b).cuda()
        xt = torch_cuda.empty_like(bt)
        A.solve(bt, xt, **sopts)
        torch_cuda.cuda.synchronize()
        assert rel_err(x, xt.cpu().numpy()) < 1e-5
    assert srv.info().solved_rhs == 8
    srv.close()
