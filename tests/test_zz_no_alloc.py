"""hm_residual_noalloc: the residual for callers that cannot allocate device
memory after start-up (for example a serving process whose memory is reserved
up front by a framework's caching allocator, where a late cudaMalloc may fail or
stall the device).  It must give the same result as hm_residual, which may grow
its workspace, using only its fixed device array; two calls in a row check that
leftovers from the previous call do not leak into the next one.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test; it also passes run alone.
"""

import ctypes

import numpy as np
import pytest

from hm_testutil import gpu_operator, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-6   # the tolerance of the other FP64-accumulated product tests


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03968_gb300 import build
    build.build()
    return torch


def _call_noalloc(A, b, x, r, n_levels):
    from paper_2307_03968_gb300 import hm
    L = hm.load()
    nrhs, n = b.shape
    norms = np.zeros(2 * nrhs)
    st = L.hm_residual_noalloc(A._h, ctypes.c_void_p(b.data_ptr()), n, ctypes.c_void_p(x.data_ptr()), n,
                               ctypes.c_void_p(r.data_ptr()), n, nrhs, n_levels,
                               norms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), hm._stream(None))
    return st, norms


def test_noalloc_residual_matches_hm_residual(torch_cuda, sphere_small):
    from oracle.hmatrix import HMatrix as OracleH
    from paper_2307_03968_gb300 import hm
    H = OracleH(sphere_small, leaf_size=32, arity=2, adm=1.0, aca_tol=1e-4)   # near + two far levels
    A = gpu_operator(H)
    rng = np.random.default_rng(31)
    for call, levels in enumerate((-1, 1)):      # two calls in a row, different level counts
        x = (rng.normal(size=(2, H.N)) + 1j * rng.normal(size=(2, H.N))).astype(np.complex64)
        b = (rng.normal(size=(2, H.N)) + 1j * rng.normal(size=(2, H.N))).astype(np.complex64)
        bt = torch_cuda.from_numpy(b).cuda()
        xt = torch_cuda.from_numpy(x).cuda()
        r_ref = torch_cuda.empty_like(bt)
        rr_ref, bb_ref = A.residual(bt, xt, r_ref, n_levels=levels)
        r_na = torch_cuda.full_like(bt, float("nan"))
        torch_cuda.cuda.synchronize()
        free0, held0 = torch_cuda.cuda.mem_get_info()[0], A.info().device_bytes
        st, norms = _call_noalloc(A, bt, xt, r_na, levels)
        assert st == hm.HM_OK, hm.load().hm_last_error()
        torch_cuda.cuda.synchronize()
        if call > 0:
            # after the first call's set-up, a call allocates nothing: neither the device's free
            # memory nor the bytes the handle holds change
            assert torch_cuda.cuda.mem_get_info()[0] == free0
            assert A.info().device_bytes == held0
        assert rel_err(r_na.cpu().numpy(), r_ref.cpu().numpy()) < TOL, call
        assert np.allclose(norms[0::2], rr_ref, rtol=TOL) and np.allclose(norms[1::2], bb_ref, rtol=TOL)


def test_noalloc_rejects_sizes_beyond_its_array(torch_cuda, sphere_small):
    from oracle.hmatrix import HMatrix as OracleH
    from paper_2307_03968_gb300 import hm
    H = OracleH(sphere_small, leaf_size=32, arity=8, adm=2.0, aca_tol=1e-4)
    A = gpu_operator(H)
    b = torch_cuda.zeros((1, H.N), dtype=torch_cuda.complex64, device="cuda")
    r = torch_cuda.empty_like(b)
    L = hm.load()
    # nrhs far beyond what 32 MiB holds for this operator: rejected before touching any buffer
    st = L.hm_residual_noalloc(A._h, ctypes.c_void_p(b.data_ptr()), H.N, ctypes.c_void_p(b.data_ptr()), H.N,
                               ctypes.c_void_p(r.data_ptr()), H.N, 5000, -1, None, hm._stream(None))
    assert st == hm.HM_ERR_ARG
    assert b"static scratch" in L.hm_last_error()
