"""Many right-hand sides in one solve: the monostatic sweep of the batched
workload (theta = 0..180 deg in 1-degree steps, phi = 0, theta-polarised,
181 right-hand sides) on the 1,920-unknown sphere, checked against the oracle
solving the same operator with the same 181 right-hand sides.

- solution: max-column relative error <= 1e-4 (the parity bar);
- monostatic RCS from both solutions (oracle far-field code): within 0.2 dB
  where the pattern is within 30 dB of its peak;
- the device right-hand sides (hm_rhs_plane_wave, operator built by hm_build)
  match the oracle's to FP32 accuracy.
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


def test_monostatic_sweep_181_rhs(torch_cuda, sphere_small):
    from synth import monostatic_sweep
    from oracle.hmatrix import HMatrix
    from oracle import series, rcs
    khat, phat = monostatic_sweep(181)
    H = HMatrix(sphere_small, leaf_size=32, arity=2, adm=1.0, aca_tol=1e-4)
    b = sphere_small.rhs(khat, phat)                       # (N, 181)
    ref = series.solve(H, b, K=2, levels=1, refine=True)   # (N, 181)
    A = gpu_operator(H)
    bt = torch_cuda.from_numpy(np.ascontiguousarray(b.T.astype(np.complex64))).cuda()
    xt = torch_cuda.empty_like(bt)
    A.solve(bt, xt, n_terms=2, n_levels=1, refine=True)
    torch_cuda.cuda.synchronize()
    x = xt.cpu().numpy()
    assert x.shape == (181, H.N)
    assert rel_err(x, ref.T) < 1e-4
    s_gpu = rcs.monostatic(sphere_small, x.T.astype(np.complex128), khat, phat)
    s_ref = rcs.monostatic(sphere_small, ref, khat, phat)
    keep = s_ref > s_ref.max() * 1e-3
    assert np.max(np.abs(rcs.db(s_gpu[keep]) - rcs.db(s_ref[keep]))) < 0.2


def test_device_plane_wave_rhs_matches_oracle(torch_cuda, sphere_small):
    from synth import icosphere, monostatic_sweep
    from paper_2307_03968_gb300.hm import HMatrix
    xyz, tri = icosphere(3, 0.3)
    A = HMatrix.build(xyz, tri, leaf_size=32, arity=8, adm=2.0, aca_tol=1e-4)
    khat, phat = monostatic_sweep(19)
    bt = torch_cuda.empty((19, A.n), dtype=torch_cuda.complex64, device="cuda")
    A.rhs_plane_wave(khat, phat, bt)
    ref = sphere_small.rhs(khat, phat).T
    assert rel_err(bt.cpu().numpy(), ref) < 1e-6
