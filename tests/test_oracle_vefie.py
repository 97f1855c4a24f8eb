"""Pins of the V-EFIE oracle (SWG basis, arxiv 2307.03968 §II eq. 4) against
results that do not come from the oracle itself:

- the SWG face enumeration against counting identities of the structured mesh;
- the analytic tetrahedron and triangle integrals against brute-force sums;
- the mass term against a closed-form Gram matrix (low-contrast limit);
- the static polarisability of homogeneous and two-layer balls against the
  textbook closed forms (interface and volume charges, normalisation);
- the bistatic RCS of a dielectric ball against the Mie series;
- the symmetry the kappa-weighted testing gives the matrix.
"""

import numpy as np
import pytest

import synth
from oracle import swg, rcs, mie


def tet_volumes(xyz, tet):
    p = xyz[tet]
    return np.abs(np.einsum('ij,ij->i', np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])) / 6.0


def equal_volume_radius(xyz, tet, mask=None):
    v = tet_volumes(xyz, tet)
    if mask is not None:
        v = v[mask]
    return (3.0 * v.sum() / (4.0 * np.pi)) ** (1.0 / 3.0)


# ------------------------------------------------------------------ basis ----

@pytest.mark.parametrize("n", [1, 2, 3])
def test_swg_faces_of_structured_cube(n):
    xyz, tet = synth.cube_tets(n, 1.0)
    fv, ft, ff = swg.swg_faces(tet)
    # 6 n^3 tetrahedra, 4 faces each: 4 nt = 2 F_int + F_bnd, F_bnd = 2 * 6 n^2
    assert len(tet) == 6 * n ** 3
    assert len(fv) == 12 * n ** 3 + 6 * n ** 2
    assert int(np.sum(ft[:, 1] < 0)) == 12 * n ** 2
    assert np.all(np.diff(fv, axis=1) > 0)                       # ascending triples
    keys = fv[:, 0].astype(np.int64) * 10 ** 12 + fv[:, 1].astype(np.int64) * 10 ** 6 + fv[:, 2]
    assert np.all(np.diff(keys) > 0)                             # sorted, unique
    inner = ft[:, 1] >= 0
    assert np.all(ft[inner, 0] < ft[inner, 1])                   # T+ = lower tetrahedron
    for f in range(len(fv)):
        for s in range(2):
            t = ft[f, s]
            if t < 0:
                continue
            cell = set(tet[t].tolist())
            assert set(fv[f].tolist()) <= cell
            assert ff[f, s] in cell and ff[f, s] not in fv[f]
    assert np.array_equal(np.bincount(ft[ft >= 0], minlength=len(tet)), np.full(len(tet), 4))


def test_ball_mesh_positive_and_conforming():
    xyz, tet = synth.ball_tets(3, 0.5)
    p = xyz[tet]
    signed = np.einsum('ij,ij->i', np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])
    assert np.all(signed > 0)
    r = np.linalg.norm(xyz, axis=1)
    assert r.max() == pytest.approx(0.5, rel=1e-12)
    # boundary faces lie on the sphere
    fv, ft, _ = swg.swg_faces(tet)
    assert np.allclose(r[fv[ft[:, 1] < 0]], 0.5)


# ------------------------------------------------------- singular integrals ----

def _tet_brute(p, r, N=160):
    """Midpoint sums of 1/R and (r'-r)/R over the tetrahedron p (4 x 3) on an
    N^3 grid of the unit reference tetrahedron, mapped affinely."""
    g = (np.arange(N) + 0.5) / N
    X, Y, Z = np.meshgrid(g, g, g, indexing='ij')
    L = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    L = L[L.sum(1) < 1.0]
    J = np.stack([p[1] - p[0], p[2] - p[0], p[3] - p[0]], 1)
    Q = p[0] + L @ J.T
    w = abs(np.linalg.det(J)) / N ** 3
    d = Q - r
    R = np.linalg.norm(d, axis=1)
    return w * np.sum(1.0 / R), w * np.sum(d / R[:, None], axis=0)


@pytest.mark.parametrize("r", [(2.0, 1.5, 0.7), (0.2, 0.2, 0.2), (0.5, 0.5, -0.3), (0.1, 0.3, 0.0)])
def test_tetrahedron_potentials_vs_brute_force(r):
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    m = swg.SWGMesh(xyz, np.array([[0, 1, 2, 3]]), 2.0)
    r = np.array(r)
    s0, s1 = m.volume_integrals(0, r)
    b0, b1 = _tet_brute(xyz, r)
    assert s0 == pytest.approx(b0, rel=2e-4)
    assert np.allclose(s1, b1, rtol=2e-4, atol=2e-5 * np.abs(b1).max())


def test_tetrahedron_potential_closed_form_at_vertex_limit():
    # Int_T 1/R dV over the unit-corner tetrahedron seen from far away -> V / |r - c|
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    m = swg.SWGMesh(xyz, np.array([[0, 1, 2, 3]]), 2.0)
    r = np.array([300.0, -200.0, 100.0])
    s0, s1 = m.volume_integrals(0, r)
    c = xyz.mean(0)
    assert s0 == pytest.approx((1 / 6) / np.linalg.norm(r - c), rel=1e-6)
    assert np.allclose(s1, (1 / 6) * (c - r) / np.linalg.norm(r - c), rtol=1e-5)


def _triangle_subdivided(p0, p1, p2, r, levels=6):
    """Sums of R and 1/R with a 3-point degree-2 rule on 4^levels congruent
    sub-triangles (converges to the integrals as the sub-triangles shrink)."""
    tris = [(p0, p1, p2)]
    for _ in range(levels):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        tris = nxt
    T = np.array(tris)                                           # (n, 3, 3)
    bary = np.array([[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]])
    Q = np.einsum('qv,tvd->tqd', bary, T)
    A = 0.5 * np.linalg.norm(np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0]), axis=1)
    R = np.linalg.norm(Q - r, axis=2)
    return np.sum(A[:, None] * R) / 3.0, np.sum(A[:, None] / R) / 3.0


@pytest.mark.parametrize("r,in_plane", [((0.3, 0.2, 0.4), False), ((0.25, 0.25, 0.0), True),
                                        ((1.5, -0.5, 0.2), False)])
def test_triangle_R_integral_vs_subdivided_quadrature(r, in_plane):
    p0, p1, p2 = np.array([0, 0, 0.0]), np.array([1.0, 0.1, 0]), np.array([0.2, 0.9, 0.0])
    r = np.array(r)
    s0, s1, sR = swg.surface_integrals(p0, p1, p2, r)
    qR, q0 = _triangle_subdivided(p0, p1, p2, r)
    assert sR == pytest.approx(qR, rel=1e-6)
    # 1/R is singular at an in-plane point: the sub-divided rule converges slowly there
    assert s0 == pytest.approx(q0, rel=2e-2 if in_plane else 1e-6)


# -------------------------------------------------------------- mass term ----

def _gram(xyz, tet, m):
    """Int f_m . f_n dV in closed form: E[lambda_i lambda_j] = (1 + delta_ij)/20
    over a tetrahedron gives Int (r-a).(r-b) = V (E|r|^2 - (a+b).c + a.b)."""
    N = m.ne
    G = np.zeros((N, N))
    vol = tet_volumes(xyz, tet)
    per_tet = [[] for _ in tet]
    for f in range(N):
        p = xyz[m.fv[f]]
        area = 0.5 * np.linalg.norm(np.cross(p[1] - p[0], p[2] - p[0]))
        for s in range(2):
            t = m.ftet[f, s]
            if t >= 0:
                per_tet[t].append((f, 1.0 if s == 0 else -1.0, xyz[m.ffree[f, s]], area))
    for t in range(len(tet)):
        p = xyz[tet[t]]
        V, c = vol[t], p.mean(0)
        Er2 = (np.sum(p * p) + np.dot(p.sum(0), p.sum(0))) / 20.0
        for (f, s, va, A) in per_tet[t]:
            for (g, sp, vb, B) in per_tet[t]:
                G[f, g] += s * sp * A * B / (9 * V) * (Er2 - np.dot(va + vb, c) + np.dot(va, vb))
    return G


def test_low_contrast_limit_is_the_gram_matrix():
    # Z = kappa/eps_r Gram + O(kappa^2): (Z/kappa - Gram/eps_r) shrinks linearly with the contrast
    xyz, tet = synth.cube_tets(2, 0.2)
    errs = []
    for d in (1e-2, 1e-3):
        er = 1.0 + d
        kap = 1.0 - 1.0 / er
        m = swg.SWGMesh(xyz, tet, er)
        G = _gram(xyz, tet, m)
        errs.append(np.linalg.norm(m.dense() / kap - G / er) / np.linalg.norm(G))
    assert errs[1] < 1e-3
    assert 0.08 < errs[1] / errs[0] < 0.12


# --------------------------------------------------- static polarisability ----

def _static_px(xyz, tet, eps):
    m = swg.SWGMesh(xyz, tet, eps)
    Z = m.dense()
    b = m.rhs(np.array([[0, 0, 1.0]]), np.array([[1.0, 0, 0]]))
    x = np.linalg.solve(Z, b[:, 0])
    return m.radiation(x, np.array([[0, 0, 1.0]]))[0][0].real


def coated_sphere_alpha(a, f, e_core, e_shell):
    """Quasi-static polarisability (per unit field, times eps0) of a two-layer
    sphere of outer radius a and core volume fraction f."""
    e1, e2 = e_core, e_shell
    return 4 * np.pi * a ** 3 * ((e2 - 1) * (e1 + 2 * e2) + f * (e1 - e2) * (1 + 2 * e2)) / \
        ((e2 + 2) * (e1 + 2 * e2) + 2 * f * (e2 - 1) * (e1 - e2))


def test_static_polarisability_homogeneous_ball():
    xyz, tet = synth.ball_tets(4, 0.002)          # k a = 0.0126: quasi-static
    a = equal_volume_radius(xyz, tet)
    for er in (2.0, 6.0):
        px = _static_px(xyz, tet, er)
        assert px == pytest.approx(4 * np.pi * a ** 3 * (er - 1) / (er + 2), rel=5e-3)


@pytest.mark.parametrize("e_core,e_shell", [(6.0, 2.0), (2.0, 6.0)])
def test_static_polarisability_two_layer_ball(e_core, e_shell):
    # the core is the image of |p|_inf <= 1/2 of the cube mesh: an interface
    # across which eps_r jumps, so the face charges kappa(T+) - kappa(T-) matter
    n = 4
    xyz, tet = synth.ball_tets(n, 0.002)
    cube, _ = synth.cube_tets(n, 2.0)
    core = np.abs(cube[tet].mean(1)).max(1) < 0.5
    a, ac = equal_volume_radius(xyz, tet), equal_volume_radius(xyz, tet, core)
    px = _static_px(xyz, tet, np.where(core, e_core, e_shell))
    ref = coated_sphere_alpha(a, (ac / a) ** 3, e_core, e_shell)
    err = abs(px / ref - 1)
    assert err < 1.5e-2
    # discriminating: the error is well below the separation of the two-layer
    # closed form from the homogeneous ball of either permittivity
    for e in (e_core, e_shell):
        sep = abs(4 * np.pi * a ** 3 * (e - 1) / (e + 2) / ref - 1)
        assert err < sep / 3, (err, sep)


# ------------------------------------------------------------ Mie, RCS ----

def test_dielectric_ball_rcs_vs_mie():
    rad, er = 0.15, 4.0
    xyz, tet = synth.ball_tets(4, rad)
    m = swg.SWGMesh(xyz, tet, er)
    b = m.rhs(np.array([[0, 0, 1.0]]), np.array([[1.0, 0, 0]]))
    x = np.linalg.solve(m.dense(), b[:, 0])
    th = np.radians([0.0, 30.0, 60.0, 120.0, 150.0, 180.0])
    got = rcs.db(rcs.bistatic_theta_pol(m, x, th))
    ref = rcs.db(mie.dielectric_bistatic_eplane(equal_volume_radius(xyz, tet), 1.0, er, th))
    assert np.abs(got - ref).max() < 0.3, got - ref


def test_dielectric_mie_series_identities():
    # lossless sphere: Q_ext = Q_sca (optical theorem); Rayleigh limit of the back-scatter
    qe, qs = mie.dielectric_efficiencies(0.2, 1.0, 4.0)
    assert qe == pytest.approx(qs, rel=1e-10)
    k, a, e = 2 * np.pi, 0.003, 4.0
    s = mie.dielectric_bistatic_eplane(a, 1.0, e, np.array([np.pi]))[0]
    assert s == pytest.approx(4 * np.pi * k ** 4 * a ** 6 * ((e - 1) / (e + 2)) ** 2, rel=1e-3)


# ------------------------------------------------------------- symmetry ----

def test_kappa_weighted_matrix_is_symmetric():
    xyz, tet = synth.cube_tets(2, 0.3)
    eps = synth.random_permittivity(len(tet), 2.0, 6.0, seed=3)
    m = swg.SWGMesh(xyz, tet, eps)
    Z = m.dense()
    scale = np.abs(Z).max()
    assert np.abs(Z - Z.T).max() < 2e-2 * scale          # quadrature breaks it only slightly
    # far pairs (no singular extraction, the same product rule both ways) are symmetric to rounding
    far_xyz, far_tet = xyz.copy(), tet.copy()
    shifted = np.concatenate([far_xyz, far_xyz + np.array([3.0, 0, 0])])
    two = np.concatenate([far_tet, far_tet + len(far_xyz)])
    m2 = swg.SWGMesh(shifted, two, np.concatenate([eps, eps[::-1]]))
    half = m.ne
    A = m2.fill(np.arange(half), np.arange(half, 2 * half))
    B = m2.fill(np.arange(half, 2 * half), np.arange(half))
    assert np.abs(A - B.T).max() < 1e-12 * np.abs(A).max()


# ------------------------------------------------------- H-Matrix on SWG ----

def test_hmatrix_of_dielectric_cube_matches_dense():
    from oracle.hmatrix import HMatrix
    xyz, tet = synth.cube_tets(4, 1.0)
    xyz = xyz * np.array([4.0, 0.5, 0.25])          # a slab, so that some cluster pairs are admissible
    eps = synth.random_permittivity(len(tet), 2.0, 6.0, seed=11)
    m = swg.SWGMesh(xyz, tet, eps)
    H = HMatrix(m, leaf_size=16, arity=2, adm=1.0, aca_tol=1e-4)
    assert len(H.far) >= 3 and sum(len(v) for v in H.far.values()) > 20
    Z = m.dense()
    # the H-Matrix mirrors the upper triangle (half storage)
    P = H.perm
    Zt = Z[np.ix_(P, P)]
    iu = np.triu_indices(m.ne, 1)
    Zs = Zt.copy()
    Zs[(iu[1], iu[0])] = Zt[iu]
    rng = np.random.default_rng(5)
    x = rng.normal(size=(m.ne, 2)) + 1j * rng.normal(size=(m.ne, 2))
    err = np.linalg.norm(H.apply(x) - Zs @ x) / np.linalg.norm(Zs @ x)
    assert err < 1e-4
