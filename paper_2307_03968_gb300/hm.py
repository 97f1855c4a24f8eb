"""ctypes binding of the hmps C ABI (include/hmps.h).

Argument marshalling only: every step of the build, factorisation and solve
runs in the CUDA library.  Device buffers are torch CUDA tensors (PyTorch is
used for device memory and streams); host buffers are numpy arrays.  The
library must be present: importing this module on a machine without the
built ``libhmps.so`` raises, there is no fallback.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhmps.so")

HM_OK, HM_ERR_ARG, HM_ERR_OOM, HM_ERR_CUDA, HM_ERR_STATE, HM_ERR_SINGULAR, HM_ERR_DIVERGED, HM_ERR_TIMEOUT = range(8)
STATUS_NAMES = ["HM_OK", "HM_ERR_ARG", "HM_ERR_OOM", "HM_ERR_CUDA", "HM_ERR_STATE", "HM_ERR_SINGULAR",
                "HM_ERR_DIVERGED", "HM_ERR_TIMEOUT"]

P = ctypes.c_void_p
I64 = ctypes.c_int64
I32 = ctypes.c_int32
PI64 = ctypes.POINTER(ctypes.c_int64)
PI32 = ctypes.POINTER(ctypes.c_int32)
PD = ctypes.POINTER(ctypes.c_double)


HM_RWG, HM_SWG = 0, 1


class HmMesh(ctypes.Structure):
    _fields_ = [("basis", ctypes.c_int), ("n_vert", I64), ("xyz", PD), ("n_cell", I64), ("cells", PI32),
                ("eps_r", PD), ("wavelength", ctypes.c_double)]


def _mesh(xyz, cells, eps_r, wavelength):
    """hm_mesh for triangles (RWG, S-EFIE) or tetrahedra with eps_r (SWG, V-EFIE);
    returns the struct and the arrays it points into (keep them alive)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    if cells.ndim != 2 or cells.shape[1] not in (3, 4):
        raise ValueError("cells must be (n, 3) triangles or (n, 4) tetrahedra")
    basis = HM_RWG if cells.shape[1] == 3 else HM_SWG
    keep = [xyz, cells]
    ep = None
    if basis == HM_SWG:
        if eps_r is None:
            raise ValueError("a tetrahedral mesh needs eps_r")
        e = np.ascontiguousarray(np.broadcast_to(np.asarray(eps_r, dtype=np.float64), (len(cells),)))
        keep.append(e)
        ep = _ptr(e, ctypes.c_double)
    m = HmMesh(basis, len(xyz), _ptr(xyz, ctypes.c_double), len(cells), _ptr(cells, ctypes.c_int32), ep, wavelength)
    return m, keep


class HmBuildOpts(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int), ("arity", ctypes.c_int), ("adm", ctypes.c_double),
                ("aca_tol", ctypes.c_double), ("levels", ctypes.c_int), ("keep_fp64", ctypes.c_int)]


class HmBlocks(ctypes.Structure):
    _fields_ = [("n", I64), ("perm", PI64), ("n_leaves", I64), ("leaf_off", PI64), ("self", PD),
                ("n_near", I64), ("near_row0", PI64), ("near_col0", PI64), ("near_m", PI32), ("near_n", PI32),
                ("near_vals", PD),
                ("n_far", I64), ("far_level", PI32), ("far_row0", PI64), ("far_col0", PI64), ("far_m", PI32),
                ("far_n", PI32), ("far_rank", PI32), ("far_u", PD), ("far_v", PD), ("keep_fp64", ctypes.c_int)]


class HmSolveOpts(ctypes.Structure):
    _fields_ = [("n_terms", ctypes.c_int), ("n_levels", ctypes.c_int), ("nested", ctypes.c_int),
                ("refine", ctypes.c_int), ("fp64", ctypes.c_int), ("graph", ctypes.c_int),
                ("persistent", ctypes.c_int)]


class HmSolveInfo(ctypes.Structure):
    _fields_ = [("rel_residual", ctypes.c_double), ("levels_used", ctypes.c_int),
                ("bytes_streamed", I64), ("kernel_launches", I64), ("norm_est", ctypes.c_double * 16),
                ("rho_est", ctypes.c_double * 16), ("convergent", ctypes.c_int)]


class HmInfo(ctypes.Structure):
    _fields_ = [("n", I64), ("n_leaves", I64), ("depth", ctypes.c_int), ("n_levels", ctypes.c_int),
                ("n_near", I64), ("n_far", I64 * 16), ("near_elems", I64), ("far_elems", I64 * 16),
                ("self_elems", I64), ("max_rank", ctypes.c_int), ("factored", ctypes.c_int),
                ("has_fp64", ctypes.c_int), ("device_bytes", I64), ("norm_est", ctypes.c_double * 16),
                ("rho_est", ctypes.c_double * 16), ("norm_iters", ctypes.c_int)]


class HmServerInfo(ctypes.Structure):
    _fields_ = [("batches", I64), ("solved_rhs", I64), ("builds", I64), ("evictions", I64),
                ("resident_bytes", I64), ("peak_resident_bytes", I64), ("loop_launches", I64),
                ("loop_stops", I64)]


EXPORTS = ["hm_build", "hm_build_from_blocks", "hm_factor_leaf", "hm_estimate_norms", "hm_powerseries_solve",
           "hm_powerseries_solve_host", "hm_apply", "hm_residual", "hm_residual_noalloc", "hm_rhs_plane_wave", "hm_profile", "hm_profile_read",
           "hm_server_create", "hm_server_create_ex", "hm_server_add_mesh", "hm_server_submit", "hm_server_wait", "hm_server_get_info",
           "hm_server_destroy",
           "hm_get_info", "hm_get_tuning", "hm_set_tuning", "hm_set_wait_limit", "hm_get_perm", "hm_get_leaves", "hm_get_blocks", "hm_get_block", "hm_sync_status",
           "hm_size", "hm_destroy", "hm_last_error", "hm_version"]

_lib = None


def load():
    """Load libhmps.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError("hmps CUDA library not built: %s is missing (run __graft_entry__.build())" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    L.hm_build.argtypes = [ctypes.POINTER(HmMesh), ctypes.POINTER(HmBuildOpts), P, ctypes.POINTER(P)]
    L.hm_build_from_blocks.argtypes = [ctypes.POINTER(HmBlocks), P, ctypes.POINTER(P)]
    L.hm_factor_leaf.argtypes = [P, P]
    L.hm_estimate_norms.argtypes = [P, ctypes.c_int, P]
    L.hm_powerseries_solve.argtypes = [P, P, I64, P, I64, ctypes.c_int, ctypes.POINTER(HmSolveOpts), P,
                                       ctypes.POINTER(HmSolveInfo)]
    L.hm_powerseries_solve_host.argtypes = [P, P, I64, P, I64, ctypes.c_int, ctypes.POINTER(HmSolveOpts), P]
    L.hm_apply.argtypes = [P, P, I64, P, I64, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
    L.hm_residual.argtypes = [P, P, I64, P, I64, P, I64, ctypes.c_int, ctypes.c_int, PD, P]
    L.hm_residual_noalloc.argtypes = [P, P, I64, P, I64, P, I64, ctypes.c_int, ctypes.c_int, PD, P]
    L.hm_rhs_plane_wave.argtypes = [P, PD, PD, ctypes.c_int, P, I64, P]
    L.hm_profile.argtypes = [P, ctypes.c_int]
    L.hm_profile_read.argtypes = [P, PD, PI64, PI64]
    L.hm_server_create.argtypes = [ctypes.c_int, I64, ctypes.c_int, ctypes.POINTER(P)]
    L.hm_server_create_ex.argtypes = [ctypes.c_int, I64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(P)]
    L.hm_server_add_mesh.argtypes = [P, ctypes.POINTER(HmMesh), ctypes.POINTER(HmBuildOpts),
                                     ctypes.POINTER(HmSolveOpts), ctypes.POINTER(ctypes.c_int), PI64]
    L.hm_server_submit.argtypes = [P, ctypes.c_int, P, I64, ctypes.c_int, PI64]
    L.hm_server_wait.argtypes = [P, I64, P, PD]
    L.hm_server_get_info.argtypes = [P, ctypes.POINTER(HmServerInfo)]
    L.hm_server_destroy.argtypes = [P]
    L.hm_server_destroy.restype = None
    L.hm_get_info.argtypes = [P, ctypes.POINTER(HmInfo)]
    L.hm_get_perm.argtypes = [P, PI64]
    L.hm_get_leaves.argtypes = [P, PI64]
    L.hm_get_tuning.argtypes = [P, ctypes.c_int, PI32, PI32, PD, PD]
    L.hm_set_tuning.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.hm_set_wait_limit.argtypes = [P, I64]
    L.hm_get_blocks.argtypes = [P, ctypes.c_int, PI64, PI64, PI64, PI32, PI32, PI32]
    L.hm_get_block.argtypes = [P, ctypes.c_int, I64, PD, PD]
    L.hm_sync_status.argtypes = [P, P]
    L.hm_size.argtypes = [P]
    L.hm_size.restype = I64
    L.hm_destroy.argtypes = [P]
    L.hm_destroy.restype = None
    L.hm_last_error.restype = ctypes.c_char_p
    L.hm_version.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name.startswith("hm_") and name not in ("hm_size", "hm_destroy", "hm_last_error", "hm_version",
                                                    "hm_server_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class HmError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))


def _check(st):
    if st != HM_OK:
        raise HmError(st, load().hm_last_error().decode())


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _stream(stream):
    if stream is None:
        import torch
        return P(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return P(stream)
    return P(stream.cuda_stream)


class HMatrix:
    """An H-Matrix operator held on the GPU (owns a hm_matrix handle)."""

    def __init__(self, handle):
        self._h = handle

    # ---- construction ------------------------------------------------------------------
    @classmethod
    def build(cls, xyz, cells, leaf_size=64, arity=8, adm=2.0, aca_tol=1e-4, levels=-1, keep_fp64=False,
              wavelength=1.0, eps_r=None, stream=None):
        """hm_build: GPU fill and ACA of the H-Matrix of a closed triangle mesh
        (RWG, S-EFIE) or of a tetrahedral mesh with per-cell eps_r (SWG, V-EFIE)."""
        mesh, _keep = _mesh(xyz, cells, eps_r, wavelength)
        opts = HmBuildOpts(leaf_size, arity, adm, aca_tol, levels, 1 if keep_fp64 else 0)
        h = P()
        _check(load().hm_build(ctypes.byref(mesh), ctypes.byref(opts), _stream(stream), ctypes.byref(h)))
        return cls(h)

    @classmethod
    def from_blocks(cls, perm, leaf_off, self_blocks, near, far, keep_fp64=False, stream=None):
        """hm_build_from_blocks.

        perm: tree position -> original index; leaf_off: leaf offsets (n_leaves+1);
        self_blocks: list of (n_i, n_i) complex arrays; near: list of
        (row0, col0, B); far: list of (level, row0, col0, U, V)."""
        n = len(perm)
        keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a

        perm_a = arr(perm, np.int64)
        lo = arr(leaf_off, np.int64)
        selfv = arr(np.concatenate([np.asarray(S, np.complex128).ravel() for S in self_blocks]), np.complex128)
        nr0 = arr([b[0] for b in near], np.int64)
        nc0 = arr([b[1] for b in near], np.int64)
        nm = arr([b[2].shape[0] for b in near], np.int32)
        nn = arr([b[2].shape[1] for b in near], np.int32)
        nv = arr(np.concatenate([np.asarray(b[2], np.complex128).ravel() for b in near])
                 if near else np.zeros(1, np.complex128), np.complex128)
        fl = arr([b[0] for b in far], np.int32)
        fr0 = arr([b[1] for b in far], np.int64)
        fc0 = arr([b[2] for b in far], np.int64)
        fm = arr([b[3].shape[0] for b in far], np.int32)
        fn = arr([b[4].shape[1] for b in far], np.int32)
        fk = arr([b[3].shape[1] for b in far], np.int32)
        fu = arr(np.concatenate([np.asarray(b[3], np.complex128).ravel() for b in far])
                 if far else np.zeros(1, np.complex128), np.complex128)
        fv = arr(np.concatenate([np.asarray(b[4], np.complex128).ravel() for b in far])
                 if far else np.zeros(1, np.complex128), np.complex128)
        B = HmBlocks(n, _ptr(perm_a, I64), len(lo) - 1, _ptr(lo, I64), _ptr(selfv.view(np.float64), ctypes.c_double),
                     len(near), _ptr(nr0, I64), _ptr(nc0, I64), _ptr(nm, I32), _ptr(nn, I32),
                     _ptr(nv.view(np.float64), ctypes.c_double),
                     len(far), _ptr(fl, I32), _ptr(fr0, I64), _ptr(fc0, I64), _ptr(fm, I32), _ptr(fn, I32),
                     _ptr(fk, I32), _ptr(fu.view(np.float64), ctypes.c_double),
                     _ptr(fv.view(np.float64), ctypes.c_double), 1 if keep_fp64 else 0)
        h = P()
        _check(load().hm_build_from_blocks(ctypes.byref(B), _stream(stream), ctypes.byref(h)))
        return cls(h)

    def factor_leaf(self, stream=None):
        _check(load().hm_factor_leaf(self._h, _stream(stream)))

    def estimate_norms(self, n_iter=32, stream=None):
        """hm_estimate_norms; returns (norm_est, rho_est) per level present (level 1 first)."""
        _check(load().hm_estimate_norms(self._h, n_iter, _stream(stream)))
        return self.norm_estimates()

    def norm_estimates(self):
        """(norm_est, rho_est) lists of the levels present, from hm_get_info."""
        i = self.info()
        nl = max(1, min(i.n_levels, 16))
        return list(i.norm_est[:nl]), list(i.rho_est[:nl])

    # ---- solve / apply -------------------------------------------------------------------
    def solve(self, b, x, n_terms=2, n_levels=1, nested=True, refine=False, fp64=False, stream=None,
              info=False, graph=True, persistent=False):
        """hm_powerseries_solve on torch CUDA tensors b, x of shape (N,) or (nrhs, N)
        (each row one right-hand side, contiguous), complex64 (complex128 if fp64);
        persistent = the one-launch solve."""
        nrhs, ldb = self._cols(b)
        _, ldx = self._cols(x)
        o = HmSolveOpts(n_terms, n_levels, 1 if nested else 0, 1 if refine else 0, 1 if fp64 else 0,
                        1 if graph else 0, 1 if persistent else 0)
        si = HmSolveInfo()
        _check(load().hm_powerseries_solve(self._h, P(b.data_ptr()), ldb, P(x.data_ptr()), ldx, nrhs,
                                           ctypes.byref(o), _stream(stream), ctypes.byref(si) if info else None))
        return si if info else None

    def solve_host(self, b, n_terms=2, n_levels=1, nested=True, refine=False, fp64=False, stream=None,
                   persistent=False, out=None):
        """hm_powerseries_solve_host on numpy arrays: b (N,) or (nrhs, N); returns x (written
        into `out` when given: a contiguous array of b's shape and dtype).  Page-locked
        arrays (for example numpy views of pinned torch tensors) are copied directly."""
        dt = np.complex128 if fp64 else np.complex64
        b = np.ascontiguousarray(b, dtype=dt)
        if out is None:
            x = np.empty_like(b)
        else:
            if out.shape != b.shape or out.dtype != b.dtype or not out.flags.c_contiguous:
                raise ValueError("out must be a contiguous array of b's shape and dtype")
            x = out
        nrhs = 1 if b.ndim == 1 else b.shape[0]
        n = b.shape[-1]
        o = HmSolveOpts(n_terms, n_levels, 1 if nested else 0, 1 if refine else 0, 1 if fp64 else 0, 1,
                        1 if persistent else 0)
        _check(load().hm_powerseries_solve_host(self._h, P(b.ctypes.data), n, P(x.ctypes.data), n, nrhs,
                                                ctypes.byref(o), _stream(stream)))
        return x

    def apply(self, x, y, n_levels=-1, fp64_accumulate=True, stream=None):
        nrhs, ldx = self._cols(x)
        _, ldy = self._cols(y)
        _check(load().hm_apply(self._h, P(x.data_ptr()), ldx, P(y.data_ptr()), ldy, nrhs, n_levels,
                               1 if fp64_accumulate else 0, _stream(stream)))

    def residual(self, b, x, r, n_levels=-1, stream=None):
        """hm_residual: r = b - A_m x (torch CUDA complex64); returns (|r|^2, |b|^2) per column."""
        nrhs, ldb = self._cols(b)
        _, ldx = self._cols(x)
        _, ldr = self._cols(r)
        norms = np.zeros(2 * max(nrhs, 1))
        _check(load().hm_residual(self._h, P(b.data_ptr()), ldb, P(x.data_ptr()), ldx, P(r.data_ptr()), ldr, nrhs,
                                  n_levels, _ptr(norms, ctypes.c_double), _stream(stream)))
        return norms[0::2], norms[1::2]

    def rhs_plane_wave(self, khat, phat, b, stream=None):
        """hm_rhs_plane_wave into the torch CUDA tensor b (nrhs, N) complex64."""
        k = np.ascontiguousarray(np.atleast_2d(khat), dtype=np.float64)
        p = np.ascontiguousarray(np.atleast_2d(phat), dtype=np.float64)
        nrhs, ldb = self._cols(b)
        assert len(k) == nrhs and len(p) == nrhs
        _check(load().hm_rhs_plane_wave(self._h, _ptr(k, ctypes.c_double), _ptr(p, ctypes.c_double), nrhs,
                                        P(b.data_ptr()), ldb, _stream(stream)))

    def profile(self, enable):
        _check(load().hm_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """(product kernel ms summed, launches, algorithmic bytes) since profile(True)."""
        ms = ctypes.c_double(0.0)
        n = I64(0)
        by = I64(0)
        _check(load().hm_profile_read(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(by)))
        return ms.value, n.value, by.value

    def sync_status(self, stream=None):
        _check(load().hm_sync_status(self._h, _stream(stream)))

    @staticmethod
    def _cols(t):
        if t.dim() == 1:
            return 1, t.shape[0]
        if not t.is_contiguous():
            raise ValueError("right-hand sides must be contiguous rows")
        return t.shape[0], t.shape[1]

    # ---- inspection ------------------------------------------------------------------------
    def info(self):
        i = HmInfo()
        _check(load().hm_get_info(self._h, ctypes.byref(i)))
        return i

    def tuning(self, nrhs):
        """hm_get_tuning: (product chunk, residual chunk, product ms, residual ms) the
        autotuner chose for nrhs right-hand sides (0 = one right-hand side at a time)."""
        a, b = ctypes.c_int32(0), ctypes.c_int32(0)
        c, d = ctypes.c_double(0), ctypes.c_double(0)
        _check(load().hm_get_tuning(self._h, nrhs, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                    ctypes.byref(d)))
        return a.value, b.value, c.value, d.value

    def set_tuning(self, nrhs, prod_rb, res_rb):
        """hm_set_tuning: pin the kernel choice for nrhs's bucket (product 1016 = tensor-core
        products; residual 1017 = owner-computes FP64-class residual)."""
        _check(load().hm_set_tuning(self._h, nrhs, prod_rb, res_rb))

    def set_wait_limit(self, polls):
        """hm_set_wait_limit: polls of each pipeline wait of the tensor-core product
        before it reports HM_ERR_TIMEOUT (negative = the default)."""
        _check(load().hm_set_wait_limit(self._h, polls))

    @property
    def n(self):
        return int(load().hm_size(self._h))

    def perm(self):
        p = np.zeros(self.n, dtype=np.int64)
        _check(load().hm_get_perm(self._h, _ptr(p, I64)))
        return p

    def leaves(self):
        lo = np.zeros(self.info().n_leaves + 1, dtype=np.int64)
        _check(load().hm_get_leaves(self._h, _ptr(lo, I64)))
        return lo

    def blocks(self, level):
        c = I64(0)
        L = load()
        _check(L.hm_get_blocks(self._h, level, ctypes.byref(c), None, None, None, None, None))
        n = c.value
        r0, c0 = np.zeros(n, np.int64), np.zeros(n, np.int64)
        m, nn, k = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int32)
        _check(L.hm_get_blocks(self._h, level, ctypes.byref(c), _ptr(r0, I64), _ptr(c0, I64), _ptr(m, I32),
                               _ptr(nn, I32), _ptr(k, I32)))
        return r0, c0, m, nn, k

    def block(self, level, index):
        r0, c0, m, n, k = self.blocks(level)
        mi, ni, ki = int(m[index]), int(n[index]), int(k[index])
        if ki == 0:
            a = np.zeros((mi, ni), np.complex128)
            _check(load().hm_get_block(self._h, level, index, _ptr(a.view(np.float64), ctypes.c_double), None))
            return a
        U = np.zeros((mi, ki), np.complex128)
        V = np.zeros((ki, ni), np.complex128)
        _check(load().hm_get_block(self._h, level, index, _ptr(U.view(np.float64), ctypes.c_double),
                                   _ptr(V.view(np.float64), ctypes.c_double)))
        return U, V

    def close(self):
        if self._h:
            load().hm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """hm_server: continuous-batching solves of several operators (complex64)."""

    def __init__(self, n_slots=4, hbm_budget_bytes=8 << 30, max_batch_rhs=64, device_loop=False):
        """device_loop: serve from a device-resident request loop (hm_server_create_ex)."""
        self._s = P()
        self.max_batch_rhs = max_batch_rhs
        _check(load().hm_server_create_ex(n_slots, hbm_budget_bytes, max_batch_rhs, 1 if device_loop else 0,
                                          ctypes.byref(self._s)))
        self._keep = []

    def add_mesh(self, xyz, cells, leaf_size=64, arity=8, adm=2.0, aca_tol=1e-4, levels=-1, wavelength=1.0,
                 n_terms=2, n_levels=1, nested=True, refine=False, eps_r=None):
        mesh, _keep = _mesh(xyz, cells, eps_r, wavelength)
        bo = HmBuildOpts(leaf_size, arity, adm, aca_tol, levels, 0)
        so = HmSolveOpts(n_terms, n_levels, 1 if nested else 0, 1 if refine else 0, 0, 1)
        op = ctypes.c_int(0)
        n = I64(0)
        _check(load().hm_server_add_mesh(self._s, ctypes.byref(mesh), ctypes.byref(bo), ctypes.byref(so),
                                         ctypes.byref(op), ctypes.byref(n)))
        return op.value, n.value

    def submit(self, op, b):
        """b: numpy (nrhs, N) or (N,); returns a request id."""
        b = np.ascontiguousarray(np.atleast_2d(b), dtype=np.complex64)
        rid = I64(0)
        _check(load().hm_server_submit(self._s, op, P(b.ctypes.data), b.shape[1], b.shape[0], ctypes.byref(rid)))
        return rid.value, b.shape

    def wait(self, req):
        rid, shape = req
        x = np.empty(shape, dtype=np.complex64)
        lat = ctypes.c_double(0.0)
        _check(load().hm_server_wait(self._s, rid, P(x.ctypes.data), ctypes.byref(lat)))
        return x, lat.value

    def info(self):
        i = HmServerInfo()
        _check(load().hm_server_get_info(self._s, ctypes.byref(i)))
        return i

    def close(self):
        if self._s:
            load().hm_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version():
    return load().hm_version().decode()
