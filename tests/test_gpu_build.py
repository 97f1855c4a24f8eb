"""GPU construction (hm_build) against the oracle.

- tree, leaves and block partition: integer work, compared bit-exactly with the
  oracle's (same documented splitting and eq. 7 rules, independent code);
- near-field blocks filled on the device (complex64) vs the oracle's complex128
  fill: elementwise, relative to the block's largest entry, <= 2e-5 (FP32
  arithmetic of the quadrature and of the analytic singular terms);
- far blocks: ACA + re-compression on the device, judged by the product U V
  against the oracle's dense block (factors are not unique): relative Frobenius
  error <= 5 x tol;
- the whole operator: hm_apply vs the oracle's own H-Matrix product, relative
  <= 5 x tol (two independent compressions of the same matrix).
"""

import numpy as np
import pytest

from hm_testutil import rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_03968_gb300 import build
    build.build()
    return torch


CASES = {
    "octree_leaf32_c2": dict(leaf_size=32, arity=8, adm=2.0),
    "binary_leaf32_c1": dict(leaf_size=32, arity=2, adm=1.0),
    "binary_leaf16_c1": dict(leaf_size=16, arity=2, adm=1.0),
}


@pytest.fixture(scope="module")
def built(torch_cuda, sphere_small):
    from synth import icosphere
    from oracle.hmatrix import HMatrix as OH
    from paper_2307_03968_gb300.hm import HMatrix
    xyz, tri = icosphere(3, 0.3)
    out = {}
    for name, kw in CASES.items():
        A = HMatrix.build(xyz, tri, aca_tol=TOL, levels=-1, **kw)
        A.factor_leaf()
        out[name] = (A, OH(sphere_small, aca_tol=TOL, **kw))
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_tree_and_partition_bit_exact(built, name):
    A, H = built[name]
    assert np.array_equal(A.perm(), H.perm)
    assert np.array_equal(A.leaves(), [0] + [o + n for (o, n) in H.leaves])
    info = A.info()
    assert info.n_levels == H.n_levels
    r0, c0, m, n, k = A.blocks(1)
    dense = k == 0
    got = sorted(zip(r0[dense], c0[dense], m[dense], n[dense]))
    want = sorted((io, jo, mm, nn) for (io, mm, jo, nn, _) in H.near)
    assert got == want
    for lev, lst in H.far.items():
        r0, c0, m, n, k = A.blocks(lev)
        lr = k > 0
        got = sorted(zip(r0[lr], c0[lr], m[lr], n[lr]))
        want = sorted((io, jo, mm, nn) for (io, mm, jo, nn, _, _) in lst)
        assert got == want, lev


def test_near_blocks_match_oracle_fill(built, sphere_small):
    A, H = built["octree_leaf32_c2"]
    P = H.perm
    r0, c0, m, n, k = A.blocks(1)
    worst = 0.0
    for idx in range(0, len(k), 97):
        if k[idx] != 0:
            continue
        B = A.block(1, idx)
        ref = sphere_small.fill(P[r0[idx]:r0[idx] + m[idx]], P[c0[idx]:c0[idx] + n[idx]])
        worst = max(worst, np.abs(B - ref).max() / np.abs(ref).max())
    assert worst < 2e-5, worst


@pytest.mark.parametrize("name", ["binary_leaf32_c1", "binary_leaf16_c1"])
def test_far_blocks_within_aca_tolerance(built, sphere_small, name):
    A, H = built[name]
    P = H.perm
    checked = 0
    for lev in range(1, A.info().n_levels + 1):
        r0, c0, m, n, k = A.blocks(lev)
        for idx in np.nonzero(k > 0)[0][::11]:
            U, V = A.block(lev, idx)
            Zb = sphere_small.fill(P[r0[idx]:r0[idx] + m[idx]], P[c0[idx]:c0[idx] + n[idx]])
            err = np.linalg.norm(U @ V - Zb) / np.linalg.norm(Zb)
            assert err < 5 * TOL, (lev, idx, err, k[idx])
            assert k[idx] < min(m[idx], n[idx])
            checked += 1
    assert checked >= 10


@pytest.mark.parametrize("name", list(CASES))
def test_operator_matches_oracle_hmatrix(torch_cuda, built, name):
    A, H = built[name]
    rng = np.random.default_rng(8)
    x = (rng.normal(size=(2, H.N)) + 1j * rng.normal(size=(2, H.N))).astype(np.complex64)
    xt = torch_cuda.from_numpy(x).cuda()
    yt = torch_cuda.empty_like(xt)
    A.apply(xt, yt, n_levels=-1, fp64_accumulate=True)
    ref = H.from_tree(H.apply(H.to_tree(x.T.astype(np.complex128)))).T
    assert rel_err(yt.cpu().numpy(), ref) < 5 * TOL


def test_build_argument_errors(torch_cuda):
    from synth import icosphere
    from paper_2307_03968_gb300.hm import HMatrix, HmError, HM_ERR_ARG
    xyz, tri = icosphere(1, 0.3)
    for kw in (dict(leaf_size=0), dict(leaf_size=5000), dict(arity=3), dict(aca_tol=0.0), dict(adm=-1.0)):
        with pytest.raises(HmError) as e:
            HMatrix.build(xyz, tri, **kw)
        assert e.value.status == HM_ERR_ARG
    bad = tri.copy()
    bad[0, 0] = len(xyz) + 5
    with pytest.raises(HmError):
        HMatrix.build(xyz, bad)
