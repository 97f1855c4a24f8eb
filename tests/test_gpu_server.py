"""Continuous-batching server (hm_server): requests for several operators of
uneven size and right-hand-side count, queued together, merged per operator
into multi-RHS solves that overlap on separate streams, with an HBM budget that
forces evictions.  Every result must equal the same request solved alone
(hm_powerseries_solve on its own handle) within 1e-5 (the sums use atomics, so
the two agree to FP32 rounding, well inside the 1e-4 parity bar)."""

import numpy as np
import pytest

from hm_testutil import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03968_gb300 import build
    build.build()
    return torch


def catalogue():
    from synth import icosphere, box_surface, closed_cylinder
    return [icosphere(3, 0.3),                                  # 1,920 unknowns
            box_surface((0.5, 0.4, 0.3), (8, 6, 5)),             # PEC box
            closed_cylinder(0.2, 0.8, 20, 10, 3)]                # closed cylinder


def test_server_mix_equals_alone(torch_cuda):
    from paper_2307_03968_gb300.hm import HMatrix, Server
    meshes = catalogue()
    opts = dict(leaf_size=32, arity=8, adm=2.0, aca_tol=1e-4)
    sopts = dict(n_terms=2, n_levels=1, refine=True)
    # operators solved alone, one handle each
    alone = []
    for xyz, tri in meshes:
        A = HMatrix.build(xyz, tri, **opts)
        A.factor_leaf()
        alone.append(A)
    sizes = [A.info().device_bytes for A in alone]          # blocks only (no solve workspace yet)
    rng = np.random.default_rng(55)
    # footprints with the workspace of a full server batch (24 right-hand sides, refinement)
    full = []
    for A in alone:
        w = torch_cuda.zeros((24, A.n), dtype=torch_cuda.complex64, device="cuda")
        A.solve(w, torch_cuda.empty_like(w), **sopts)
        full.append(A.info().device_bytes)
    torch_cuda.cuda.synchronize()
    # budget below the sum of all operators: the server must evict to serve them
    srv = Server(n_slots=3, hbm_budget_bytes=int(max(sizes) * 1.3), max_batch_rhs=24)
    ops = [srv.add_mesh(xyz, tri, **opts, **sopts) for xyz, tri in meshes]
    for (op, n), A in zip(ops, alone):
        assert n == A.n
    reqs = []
    for q in range(40):
        k = int(rng.integers(len(meshes)))
        op, n = ops[k]
        nrhs = int(rng.integers(1, 9))
        b = (rng.normal(size=(nrhs, n)) + 1j * rng.normal(size=(nrhs, n))).astype(np.complex64)
        reqs.append((k, b, srv.submit(op, b)))
    lat = []
    for k, b, r in reqs:
        x, ms = srv.wait(r)
        lat.append(ms)
        bt = torch_cuda.from_numpy(b).cuda()
        xt = torch_cuda.empty_like(bt)
        alone[k].solve(bt, xt, **sopts)
        torch_cuda.cuda.synchronize()
        assert rel_err(x, xt.cpu().numpy()) < 1e-5
    info = srv.info()
    assert info.solved_rhs == sum(b.shape[0] for _, b, _ in reqs)
    assert info.batches < len(reqs)          # requests were merged
    assert all(v > 0 for v in lat)
    # one request at a time, cycling through the operators: each one is idle when
    # the next is built, so the budget must evict it (and rebuild it later)
    for rnd in range(2):
        for k, (op, n) in enumerate(ops):
            b = (rng.normal(size=(1, n)) + 1j * rng.normal(size=(1, n))).astype(np.complex64)
            x, _ = srv.wait(srv.submit(op, b))
            bt = torch_cuda.from_numpy(b).cuda()
            xt = torch_cuda.empty_like(bt)
            alone[k].solve(bt, xt, **sopts)
            torch_cuda.cuda.synchronize()
            assert rel_err(x, xt.cpu().numpy()) < 1e-5
    info = srv.info()
    assert info.evictions >= len(meshes) and info.builds >= 2 * len(meshes)
    # at most the two largest operators (each with its workspace) resident at once
    assert info.peak_resident_bytes <= 1.3 * (sorted(full)[-1] + sorted(full)[-2])
    srv.close()


def test_server_rejects_bad_requests(torch_cuda):
    from synth import icosphere
    from paper_2307_03968_gb300.hm import Server, HmError, HM_ERR_ARG
    srv = Server(n_slots=1, hbm_budget_bytes=1 << 30, max_batch_rhs=4)
    xyz, tri = icosphere(2, 0.15)
    op, n = srv.add_mesh(xyz, tri, leaf_size=32)
    with pytest.raises(HmError) as e:
        srv.submit(op, np.zeros((1, n + 1), np.complex64))
    assert e.value.status == HM_ERR_ARG
    with pytest.raises(HmError):
        srv.submit(op, np.zeros((5, n), np.complex64))       # more than max_batch_rhs
    with pytest.raises(HmError):
        srv.submit(op + 7, np.zeros((1, n), np.complex64))
    srv.close()
