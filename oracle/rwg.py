"""RWG basis on a closed triangle mesh and the ctypes wrapper of efie.c.

Oracle — test infrastructure only.

RWG functions (ref. [20] of arxiv 2307.03968, used in §II): one unknown per
interior edge, supported on the two triangles T+ and T- sharing it.  Ordering
(the "original unknown order" of the whole build): edges sorted by
(min vertex id, max vertex id); T+ is the triangle with the lower index.
"""

import ctypes
import os
import subprocess
import numpy as np

ETA0 = 376.730313461770655   # free-space impedance (ohm) = mu0 * c0
_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_DIR = os.path.join(_HERE, "_lib")
_LIB_PATH = os.path.join(_LIB_DIR, "libhmoracle.so")
_SRCS = [os.path.join(_HERE, "efie.c"), os.path.join(_HERE, "vefie.c")]
_lib = None


def build_lib(force=False):
    """Compile efie.c and vefie.c into oracle/_lib/libhmoracle.so (gcc, OpenMP)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
                           "-ffp-contract=off", *_SRCS, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build_lib())
        P = ctypes.c_void_p
        L.hmo_ctx_new.restype = P
        L.hmo_ctx_new.argtypes = [ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int, P, P, P,
                                  ctypes.c_double, ctypes.c_double]
        L.hmo_ctx_free.argtypes = [P]
        L.hmo_fill.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int, P]
        L.hmo_rhs.argtypes = [P, ctypes.c_int, P, P, P]
        L.hmo_radiation.argtypes = [P, P, ctypes.c_int, P, P]
        L.hmo_potential_integrals.argtypes = [P, P, P, P, P, P]
        L.hmo_quad_rule.argtypes = [P, P]
        L.hmo_aca.restype = ctypes.c_int
        L.hmo_aca.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int, ctypes.c_double, ctypes.c_int, P, P]
        L.hmo_aca_many.argtypes = [P, ctypes.c_int, P, P, P, P, P, ctypes.c_double, P, P, P, P, P, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def rwg_edges(tri):
    """Interior edges of a triangle mesh as RWG unknowns.

    Returns (edge_vertices (ne,2), edge_tri (ne,2) = (T+, T-),
    edge_free (ne,2) = free vertex of T+ and of T-), all int32, sorted by
    (min vertex, max vertex).  Edges not shared by exactly two triangles carry
    no RWG function and are skipped."""
    owners = {}
    for t, (a, b, c) in enumerate(tri.tolist()):
        for (u, v, w) in ((a, b, c), (b, c, a), (c, a, b)):
            key = (u, v) if u < v else (v, u)
            owners.setdefault(key, []).append((t, w))
    keys = sorted(k for k, o in owners.items() if len(o) == 2)
    ev = np.array(keys, dtype=np.int32).reshape(-1, 2)
    et = np.zeros_like(ev)
    ef = np.zeros_like(ev)
    for i, key in enumerate(keys):
        (t0, w0), (t1, w1) = sorted(owners[key])
        et[i] = (t0, t1)
        ef[i] = (w0, w1)
    return ev, et, ef


class RWGMesh:
    """A triangle mesh with its RWG basis and a handle on the C entry code."""

    def __init__(self, xyz, tri, wavelength=1.0):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.ev, self.etri, self.efree = rwg_edges(self.tri)
        self.ne = len(self.ev)
        self.elen = np.ascontiguousarray(
            np.linalg.norm(self.xyz[self.ev[:, 0]] - self.xyz[self.ev[:, 1]], axis=1))
        self.k = 2.0 * np.pi / wavelength
        self.eta = ETA0
        # sigma = rcs_scale |p . F|^2 for the radiation vector F below
        self.rcs_scale = (self.k * self.eta) ** 2 / (4.0 * np.pi)
        self._ctx = lib().hmo_ctx_new(len(self.xyz), _p(self.xyz), len(self.tri), _p(self.tri),
                                      self.ne, _p(self.etri), _p(self.efree), _p(self.elen),
                                      self.k, self.eta)

    def __del__(self):
        if getattr(self, "_ctx", None) and _lib is not None:
            _lib.hmo_ctx_free(self._ctx)
            self._ctx = None

    # --- geometry used by the tree ------------------------------------------------
    def centres(self):
        """Edge midpoints: the point each unknown is sorted by in the tree."""
        return 0.5 * (self.xyz[self.ev[:, 0]] + self.xyz[self.ev[:, 1]])

    def support_boxes(self):
        """Axis-aligned box of the four vertices of T+ and T- of each unknown."""
        v = np.concatenate([self.ev, self.efree], axis=1)
        p = self.xyz[v]                       # (ne, 4, 3)
        return p.min(axis=1), p.max(axis=1)

    # --- matrix entries -------------------------------------------------------------
    def fill(self, rows, cols):
        """Dense Z[rows][:, cols] (complex128), entry by entry."""
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        out = np.empty((len(rows), len(cols)), dtype=np.complex128)
        if out.size:
            lib().hmo_fill(self._ctx, _p(rows), len(rows), _p(cols), len(cols), _p(out))
        return out

    def dense(self):
        idx = np.arange(self.ne, dtype=np.int32)
        return self.fill(idx, idx)

    def rhs(self, khat, phat):
        """b (ne, R): b_m = Int f_m . p_hat exp(-jk k_hat.r) dS for each plane wave."""
        khat = np.ascontiguousarray(np.atleast_2d(khat), dtype=np.float64)
        phat = np.ascontiguousarray(np.atleast_2d(phat), dtype=np.float64)
        b = np.empty((len(khat), self.ne), dtype=np.complex128)
        lib().hmo_rhs(self._ctx, len(khat), _p(khat), _p(phat), _p(b))
        return np.ascontiguousarray(b.T)

    def radiation(self, x, rhat):
        """F(r_hat) = Int J exp(+jk r_hat.r') dS' for J = sum x_n f_n; (ndir, 3)."""
        x = np.ascontiguousarray(x, dtype=np.complex128)
        rhat = np.ascontiguousarray(np.atleast_2d(rhat), dtype=np.float64)
        F = np.empty((len(rhat), 3), dtype=np.complex128)
        lib().hmo_radiation(self._ctx, _p(x), len(rhat), _p(rhat), _p(F))
        return F

    def aca(self, rows, cols, tol, kmax=None):
        """Raw ACA factors (U (m,k), V (k,n)) of Z[rows][:, cols]."""
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        m, n = len(rows), len(cols)
        kmax = min(m, n) if kmax is None else min(kmax, m, n)
        U = np.zeros(kmax * m, dtype=np.complex128)
        V = np.zeros(kmax * n, dtype=np.complex128)
        k = lib().hmo_aca(self._ctx, _p(rows), m, _p(cols), n, tol, kmax, _p(U), _p(V))
        return U[:k * m].reshape(k, m).T.copy(), V[:k * n].reshape(k, n).copy()

    def aca_many(self, blocks, tol):
        """ACA of many blocks [(rows, cols), ...] in parallel (OpenMP)."""
        nb = len(blocks)
        if nb == 0:
            return []
        idx = np.concatenate([np.concatenate([r, c]) for r, c in blocks]).astype(np.int32)
        m = np.array([len(r) for r, _ in blocks], dtype=np.int32)
        n = np.array([len(c) for _, c in blocks], dtype=np.int32)
        sizes = m.astype(np.int64) + n
        roff = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        coff = roff + m
        kmax = np.minimum(m, n).astype(np.int32)
        usz = kmax.astype(np.int64) * m
        vsz = kmax.astype(np.int64) * n
        uoff = np.concatenate([[0], np.cumsum(usz)[:-1]]).astype(np.int64)
        voff = np.concatenate([[0], np.cumsum(vsz)[:-1]]).astype(np.int64)
        U = np.zeros(int(usz.sum()), dtype=np.complex128)
        V = np.zeros(int(vsz.sum()), dtype=np.complex128)
        rank = np.zeros(nb, dtype=np.int32)
        lib().hmo_aca_many(self._ctx, nb, _p(idx), _p(roff), _p(m), _p(coff), _p(n), tol,
                           _p(kmax), _p(uoff), _p(voff), _p(U), _p(V), _p(rank))
        out = []
        for b in range(nb):
            k, mb, nb_ = int(rank[b]), int(m[b]), int(n[b])
            Ub = U[uoff[b]:uoff[b] + k * mb].reshape(k, mb).T.copy()
            Vb = V[voff[b]:voff[b] + k * nb_].reshape(k, nb_).copy()
            out.append((Ub, Vb))
        return out


def quad_rule():
    """(barycentric points (7, 3), weights (7,)) of the C code's triangle rule."""
    bary = np.zeros((7, 3))
    w = np.zeros(7)
    lib().hmo_quad_rule(_p(bary), _p(w))
    return bary, w


def potential_integrals(p0, p1, p2, r):
    """(Int_T 1/R dS', Int_T (rho'-rho)/R dS') of the C code, for tests."""
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (p0, p1, p2, r)]
    s0 = np.zeros(1)
    s1 = np.zeros(3)
    lib().hmo_potential_integrals(*[_p(v) for v in a], _p(s0), _p(s1))
    return s0[0], s1
