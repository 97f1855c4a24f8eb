"""SWG basis on a tetrahedral mesh and the ctypes wrapper of vefie.c.

Oracle — test infrastructure only.

SWG functions (ref. [21] of arxiv 2307.03968, the volume basis of the V-EFIE,
eq. 4): one unknown per face of the tetrahedral mesh, supported on the one or
two tetrahedra sharing it.  Ordering (the "original unknown order" of the
volume solver): faces sorted by their ascending vertex triple; T+ is the
tetrahedron with the lower index; a boundary face has T- = -1.
"""

import ctypes
import numpy as np

from .rwg import lib as _rwg_lib, _p

_vlib = None


def lib():
    global _vlib
    if _vlib is None:
        L = _rwg_lib()
        P = ctypes.c_void_p
        L.vmo_ctx_new.restype = P
        L.vmo_ctx_new.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, ctypes.c_int, P, P, P, ctypes.c_double]
        L.vmo_ctx_free.argtypes = [P]
        L.vmo_fill.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int, P]
        L.vmo_rhs.argtypes = [P, ctypes.c_int, P, P, P]
        L.vmo_radiation.argtypes = [P, P, ctypes.c_int, P, P]
        L.vmo_volume_integrals.argtypes = [P, ctypes.c_int, P, P, P]
        L.hmo_potential_integrals3.argtypes = [P, P, P, P, P, P, P]
        L.vmo_aca.restype = ctypes.c_int
        L.vmo_aca.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int, ctypes.c_double, ctypes.c_int, P, P]
        L.vmo_aca_many.argtypes = [P, ctypes.c_int, P, P, P, P, P, ctypes.c_double, P, P, P, P, P, P]
        _vlib = L
    return _vlib


def swg_faces(tet):
    """Faces of a tetrahedral mesh as SWG unknowns.

    Returns (face_vertices (nf,3) ascending, face_tet (nf,2) = (T+, T-),
    face_free (nf,2) = vertex of T+ and of T- opposite the face), int32,
    sorted by the vertex triple.  Boundary faces have T- = -1 and free -1."""
    tet = np.asarray(tet, dtype=np.int64)
    nt = len(tet)
    keys = []
    for o in range(4):
        cols = [c for c in range(4) if c != o]
        keys.append(np.sort(tet[:, cols], axis=1))
    K = np.concatenate(keys)                                   # (4 nt, 3), tet-major within each o
    owner = np.tile(np.arange(nt), 4)
    free = np.concatenate([tet[:, o] for o in range(4)])
    order = np.lexsort((owner, K[:, 2], K[:, 1], K[:, 0]))     # by triple, then owner
    K, owner, free = K[order], owner[order], free[order]
    new = np.ones(len(K), dtype=bool)
    new[1:] = np.any(K[1:] != K[:-1], axis=1)
    start = np.flatnonzero(new)
    cnt = np.diff(np.append(start, len(K)))
    if np.any(cnt > 2):
        raise ValueError("non-manifold tetrahedral mesh: a face is shared by more than two tetrahedra")
    fv = K[start].astype(np.int32)
    ft = np.full((len(start), 2), -1, dtype=np.int32)
    ff = np.full((len(start), 2), -1, dtype=np.int32)
    ft[:, 0], ff[:, 0] = owner[start], free[start]
    two = cnt == 2
    ft[two, 1], ff[two, 1] = owner[start[two] + 1], free[start[two] + 1]
    return fv, ft, ff


class SWGMesh:
    """A tetrahedral mesh with per-tetrahedron relative permittivity, its SWG
    basis and a handle on the C entry code."""

    def __init__(self, xyz, tet, eps_r, wavelength=1.0):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.tet = np.ascontiguousarray(tet, dtype=np.int32)
        self.eps_r = np.ascontiguousarray(np.broadcast_to(np.asarray(eps_r, dtype=np.float64),
                                                          (len(self.tet),)))
        self.fv, self.ftet, self.ffree = swg_faces(self.tet)
        self.ne = len(self.fv)                  # unknown count (same name as the RWG mesh)
        self.k = 2.0 * np.pi / wavelength
        # sigma = k^4 / (4 pi) |p . P|^2 for the radiation vector P below
        self.rcs_scale = self.k ** 4 / (4.0 * np.pi)
        self._ctx = lib().vmo_ctx_new(len(self.xyz), _p(self.xyz), len(self.tet), _p(self.tet),
                                      _p(self.eps_r), self.ne, _p(self.ftet), _p(self.ffree), _p(self.fv),
                                      self.k)

    def __del__(self):
        if getattr(self, "_ctx", None) and _vlib is not None:
            _vlib.vmo_ctx_free(self._ctx)
            self._ctx = None

    # --- geometry used by the tree ------------------------------------------------
    def centres(self):
        """Face centroids (sum of the three vertices in ascending id order, / 3)."""
        p = self.xyz[self.fv]
        return (p[:, 0] + p[:, 1] + p[:, 2]) / 3.0

    def support_boxes(self):
        """Axis-aligned box of the vertices of T+ and T- of each unknown."""
        p = self.xyz[self.fv]                                   # (nf, 3, 3)
        f0 = self.xyz[self.ffree[:, 0]]
        f1 = np.where((self.ffree[:, 1] >= 0)[:, None], self.xyz[np.maximum(self.ffree[:, 1], 0)], f0)
        allp = np.concatenate([p, f0[:, None], f1[:, None]], axis=1)
        return allp.min(axis=1), allp.max(axis=1)

    # --- matrix entries -------------------------------------------------------------
    def fill(self, rows, cols):
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        out = np.empty((len(rows), len(cols)), dtype=np.complex128)
        if out.size:
            lib().vmo_fill(self._ctx, _p(rows), len(rows), _p(cols), len(cols), _p(out))
        return out

    def dense(self):
        idx = np.arange(self.ne, dtype=np.int32)
        return self.fill(idx, idx)

    def rhs(self, khat, phat):
        """b (nf, R): b_m = Int kappa f_m . p_hat exp(-jk k_hat.r) dV."""
        khat = np.ascontiguousarray(np.atleast_2d(khat), dtype=np.float64)
        phat = np.ascontiguousarray(np.atleast_2d(phat), dtype=np.float64)
        b = np.empty((len(khat), self.ne), dtype=np.complex128)
        lib().vmo_rhs(self._ctx, len(khat), _p(khat), _p(phat), _p(b))
        return np.ascontiguousarray(b.T)

    def radiation(self, x, rhat):
        """P(r_hat) = Int kappa D/eps0 exp(+jk r_hat.r') dV' for D = eps0 sum x_n f_n; (ndir, 3)."""
        x = np.ascontiguousarray(x, dtype=np.complex128)
        rhat = np.ascontiguousarray(np.atleast_2d(rhat), dtype=np.float64)
        P = np.empty((len(rhat), 3), dtype=np.complex128)
        lib().vmo_radiation(self._ctx, _p(x), len(rhat), _p(rhat), _p(P))
        return P

    def aca(self, rows, cols, tol, kmax=None):
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        m, n = len(rows), len(cols)
        kmax = min(m, n) if kmax is None else min(kmax, m, n)
        U = np.zeros(kmax * m, dtype=np.complex128)
        V = np.zeros(kmax * n, dtype=np.complex128)
        k = lib().vmo_aca(self._ctx, _p(rows), m, _p(cols), n, tol, kmax, _p(U), _p(V))
        return U[:k * m].reshape(k, m).T.copy(), V[:k * n].reshape(k, n).copy()

    def aca_many(self, blocks, tol):
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
        lib().vmo_aca_many(self._ctx, nb, _p(idx), _p(roff), _p(m), _p(coff), _p(n), tol,
                           _p(kmax), _p(uoff), _p(voff), _p(U), _p(V), _p(rank))
        out = []
        for b in range(nb):
            k, mb, nb_ = int(rank[b]), int(m[b]), int(n[b])
            out.append((U[uoff[b]:uoff[b] + k * mb].reshape(k, mb).T.copy(),
                        V[voff[b]:voff[b] + k * nb_].reshape(k, nb_).copy()))
        return out

    # --- pieces exposed for the pins --------------------------------------------------
    def volume_integrals(self, t, r):
        """(Int_T 1/R dV', Int_T (r'-r)/R dV') of the C code for tetrahedron t."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        s0 = np.zeros(1)
        s1 = np.zeros(3)
        lib().vmo_volume_integrals(self._ctx, int(t), _p(r), _p(s0), _p(s1))
        return s0[0], s1


def surface_integrals(p0, p1, p2, r):
    """(Int 1/R dS', Int (rho'-rho)/R dS', Int R dS') over a triangle, for tests."""
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (p0, p1, p2, r)]
    s0, s1, sR = np.zeros(1), np.zeros(3), np.zeros(1)
    lib().hmo_potential_integrals3(*[_p(v) for v in a], _p(s0), _p(s1), _p(sR))
    return s0[0], s1, sR[0]
