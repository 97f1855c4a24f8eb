"""The device-resident request loop (hm_server_create_ex with device_loop = 1):
one cooperative kernel stays on the GPU and serves the batches posted to a ring
in mapped host memory.  Every result must equal the same request solved alone
(hm_powerseries_solve on its own handle) within 1e-5, as for the host-scheduled
server; the loop must survive going idle (it leaves by itself and is launched
again by the next batch) and a budget that forces evictions (builds stop it)."""

import time

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


def _alone(torch_cuda, A, b, sopts):
    bt = torch_cuda.from_numpy(b).cuda()
    xt = torch_cuda.empty_like(bt)
    A.solve(bt, xt, **sopts)
    torch_cuda.cuda.synchronize()
    return xt.cpu().numpy()


def test_device_loop_mix_equals_alone(torch_cuda):
    from synth import icosphere, box_surface, closed_cylinder
    from paper_2307_03968_gb300.hm import HMatrix, Server
    meshes = [icosphere(3, 0.3), box_surface((0.5, 0.4, 0.3), (8, 6, 5)), closed_cylinder(0.2, 0.8, 20, 10, 3)]
    opts = dict(leaf_size=32, arity=8, adm=2.0, aca_tol=1e-4)
    sopts = dict(n_terms=2, n_levels=1, refine=True)
    alone = []
    for xyz, tri in meshes:
        A = HMatrix.build(xyz, tri, **opts)
        A.factor_leaf()
        alone.append(A)
    sizes = [A.info().device_bytes for A in alone]
    srv = Server(n_slots=3, hbm_budget_bytes=int(max(sizes) * 1.3), max_batch_rhs=24, device_loop=True)
    ops = [srv.add_mesh(xyz, tri, **opts, **sopts) for xyz, tri in meshes]
    rng = np.random.default_rng(57)
    reqs = []
    for q in range(30):
        k = int(rng.integers(len(meshes)))
        op, n = ops[k]
        nrhs = int(rng.integers(1, 9))
        b = (rng.normal(size=(nrhs, n)) + 1j * rng.normal(size=(nrhs, n))).astype(np.complex64)
        reqs.append((k, b, srv.submit(op, b)))
    for k, b, r in reqs:
        x, ms = srv.wait(r)
        assert ms > 0
        assert rel_err(x, _alone(torch_cuda, alone[k], b, sopts)) < 1e-5
    info = srv.info()
    assert info.loop_launches >= 1 and info.batches < len(reqs)
    # one request at a time, cycling through the operators: each one is idle when the
    # next is built, so the budget (about one operator) must evict it; builds stop the loop
    for rnd in range(2):
        for k, (op, n) in enumerate(ops):
            b = (rng.normal(size=(2, n)) + 1j * rng.normal(size=(2, n))).astype(np.complex64)
            x, _ = srv.wait(srv.submit(op, b))
            assert rel_err(x, _alone(torch_cuda, alone[k], b, sopts)) < 1e-5
    info = srv.info()
    assert info.evictions >= len(meshes) and info.loop_stops >= len(meshes)
    # idle: the loop leaves by itself after about a second; the next batch launches it again
    time.sleep(2.5)
    launches = srv.info().loop_launches
    op, n = ops[0]
    b = (rng.normal(size=(3, n)) + 1j * rng.normal(size=(3, n))).astype(np.complex64)
    x, _ = srv.wait(srv.submit(op, b))
    assert rel_err(x, _alone(torch_cuda, alone[0], b, sopts)) < 1e-5
    assert srv.info().loop_launches == launches + 1
    srv.close()
