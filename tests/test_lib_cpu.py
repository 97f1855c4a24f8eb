"""CPU-side checks of the CUDA library: it loads, exports every entry point
declared in include/hmps.h, and rejects bad arguments on the host before any
device work (no GPU needed for these calls)."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2307_03968_gb300 import build as B
    B.build()
    from paper_2307_03968_gb300 import hm
    return hm.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "hmps.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hm_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    from paper_2307_03968_gb300 import hm
    assert sorted(hm.EXPORTS) == names


def test_version_and_last_error(lib):
    from paper_2307_03968_gb300 import hm
    assert "sm_103a" in hm.version()


def test_host_argument_errors(lib):
    from paper_2307_03968_gb300 import hm
    out = ctypes.c_void_p()
    assert lib.hm_build_from_blocks(None, None, ctypes.byref(out)) == hm.HM_ERR_ARG
    assert b"null" in lib.hm_last_error()
    B = hm.HmBlocks()
    B.n = 0
    assert lib.hm_build_from_blocks(ctypes.byref(B), None, ctypes.byref(out)) == hm.HM_ERR_ARG
    assert lib.hm_factor_leaf(None, None) == hm.HM_ERR_ARG
    assert lib.hm_estimate_norms(None, 32, None) == hm.HM_ERR_ARG
    o = hm.HmSolveOpts(2, 1, 1, 0, 0, 0)
    assert lib.hm_powerseries_solve(None, None, 0, None, 0, 1, ctypes.byref(o), None, None) == hm.HM_ERR_ARG
    assert lib.hm_apply(None, None, 0, None, 0, 1, 1, 1, None) == hm.HM_ERR_ARG
    assert lib.hm_size(None) == 0
    lib.hm_destroy(None)


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    from paper_2307_03968_gb300 import hm
    monkeypatch.setattr(hm, "_lib", None)
    monkeypatch.setattr(hm, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(OSError):
        hm.load()


def test_build_rejects_bad_meshes_on_the_host(lib):
    """hm_build validates the mesh before any device work."""
    import synth
    from paper_2307_03968_gb300 import hm
    xyz, tet = synth.cube_tets(1, 1.0)
    opts = hm.HmBuildOpts(16, 2, 1.0, 1e-4, -1, 0)
    out = ctypes.c_void_p()

    def status(xyz, cells, eps):
        m, keep = hm._mesh(xyz, cells, eps, 1.0)
        return lib.hm_build(ctypes.byref(m), ctypes.byref(opts), None, ctypes.byref(out))

    bad = tet.copy()
    bad[0, 0] = len(xyz) + 3
    assert status(xyz, bad, 2.0) == hm.HM_ERR_ARG                      # vertex id out of range
    assert status(xyz, tet, -1.0) == hm.HM_ERR_ARG                     # eps_r must be > 0
    assert status(xyz, tet, np.nan) == hm.HM_ERR_ARG
    rep = tet.copy()
    rep[0, 1] = rep[0, 0]
    assert status(xyz, rep, 2.0) == hm.HM_ERR_ARG                      # repeated vertex
    three = np.concatenate([tet, tet[:1]])                             # a face of three tetrahedra
    assert status(xyz, three, 2.0) == hm.HM_ERR_ARG
    flat = xyz.copy()
    flat[:, 2] = 0.0                                                   # zero-volume tetrahedra
    assert status(flat, tet, 2.0) == hm.HM_ERR_ARG
    m, keep = hm._mesh(xyz, tet, 2.0, 1.0)
    m.eps_r = None
    assert lib.hm_build(ctypes.byref(m), ctypes.byref(opts), None, ctypes.byref(out)) == hm.HM_ERR_ARG
    assert b"eps_r" in lib.hm_last_error()
    tri_bad = np.array([[0, 1, 99], [1, 2, 3]], dtype=np.int32)
    assert status(xyz, tri_bad, None) == hm.HM_ERR_ARG                 # triangle id out of range
    with pytest.raises(ValueError):
        hm._mesh(xyz, tet, None, 1.0)                                  # tetrahedra need eps_r
