"""Pins of the oracle's EFIE discretisation against closed forms and physics.

- the triangle rule integrates every monomial of degree <= 5 exactly;
- the analytic 1/R potential integrals equal independent numerical integrals
  (fine subdivision off the triangle, polar integration for in-plane points);
- the RCS of the MoM solution of a PEC sphere matches the Mie series;
- the Mie series itself satisfies the optical theorem and the Rayleigh limit;
- the Galerkin matrix is complex symmetric up to quadrature error, so the
  half-storage mirror of §III changes it only at that level.
"""

import math

import numpy as np
import pytest

from oracle import mie, rcs
from oracle.rwg import potential_integrals, quad_rule, rwg_edges


def test_quadrature_rule_exact_to_degree_5():
    bary, w = quad_rule()
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(bary.sum(axis=1), 1.0, atol=1e-15)
    # reference triangle (0,0),(1,0),(0,1): int x^a y^b = a! b! / (a+b+2)!, area 1/2
    x, y = bary[:, 1], bary[:, 2]
    for a in range(6):
        for b in range(6 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            got = 0.5 * np.sum(w * x ** a * y ** b)
            assert abs(got - exact) < 1e-15, (a, b)
    # and is not exact at degree 6 (it is a degree-5 rule)
    got = 0.5 * np.sum(w * x ** 6)
    assert abs(got - math.factorial(6) / math.factorial(8)) > 1e-6


def _subdivision_integrals(p0, p1, p2, r, n=500):
    e1, e2 = p1 - p0, p2 - p0
    nrm = np.cross(e1, e2)
    area = 0.5 * np.linalg.norm(nrm)
    nrm /= np.linalg.norm(nrm)
    rho = r - (nrm @ (r - p0)) * nrm
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    up = i + j < n
    dn = i + j < n - 1
    u = np.concatenate([(i[up] + 1 / 3) / n, (i[dn] + 2 / 3) / n])
    v = np.concatenate([(j[up] + 1 / 3) / n, (j[dn] + 2 / 3) / n])
    P = p0 + u[:, None] * e1 + v[:, None] * e2
    R = np.linalg.norm(P - r, axis=1)
    w = area / (n * n)
    return w * np.sum(1 / R), w * ((P - rho) / R[:, None]).sum(axis=0)


TRI = (np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.1, 0.0]), np.array([0.3, 0.9, 0.05]))


@pytest.mark.parametrize("r", [[0.4, 0.3, 0.5], [2.0, 1.0, 0.3], [1.5, 1.2, 0.0], [-0.5, 0.2, 0.2]])
def test_potential_integrals_off_triangle(r):
    r = np.array(r)
    s0, s1 = potential_integrals(*TRI, r)
    b0, b1 = _subdivision_integrals(*TRI, r)
    assert abs(s0 - b0) < 1e-5 * abs(b0)
    assert np.linalg.norm(s1 - b1) < 1e-5 * np.linalg.norm(b1)


def test_potential_integral_in_plane_interior_point_polar():
    # For a point inside the triangle and in its plane, int 1/R dS = int_0^2pi rho_max(phi) dphi.
    p0, p1, p2 = (np.array(v, dtype=float) for v in ([0, 0, 0], [1, 0, 0], [0.2, 0.8, 0]))
    r = np.array([0.35, 0.25, 0.0])
    s0, s1 = potential_integrals(p0, p1, p2, r)
    nphi = 200000
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    d = np.stack([np.cos(phi), np.sin(phi)], axis=1)
    rmax = np.full(nphi, np.inf)
    verts = [p0[:2], p1[:2], p2[:2]]
    for k in range(3):
        a, b = verts[k], verts[(k + 1) % 3]
        e = b - a
        # solve r + t d = a + s e  for t >= 0, 0 <= s <= 1
        den = d[:, 0] * (-e[1]) - d[:, 1] * (-e[0])
        rhs = a - r[:2]
        t = (rhs[0] * (-e[1]) - rhs[1] * (-e[0])) / den
        s = (d[:, 0] * rhs[1] - d[:, 1] * rhs[0]) / den
        ok = (t > 0) & (s >= 0) & (s <= 1)
        rmax = np.where(ok & (t < rmax), t, rmax)
    polar0 = np.sum(rmax) * 2 * np.pi / nphi
    # int (rho'-rho)/R dS = int_0^2pi d(phi) rho_max^2 / 2 (unit direction)
    polar1 = (d * (rmax ** 2 / 2)[:, None]).sum(axis=0) * 2 * np.pi / nphi
    assert abs(s0 - polar0) < 1e-7 * polar0
    assert np.linalg.norm(s1[:2] - polar1) < 1e-6 * np.linalg.norm(polar1)
    assert abs(s1[2]) < 1e-14


def test_rwg_edges_closed_mesh(sphere_small):
    m = sphere_small
    assert m.ne == 1920
    # every triangle edge of a closed mesh is interior; T+ < T-
    assert np.all(m.etri[:, 0] < m.etri[:, 1])
    for e in range(0, m.ne, 97):
        a, b = m.ev[e]
        for s in range(2):
            t = m.tri[m.etri[e, s]]
            assert a in t and b in t and m.efree[e, s] in t and m.efree[e, s] not in (a, b)


def test_rwg_edges_open_mesh_skips_boundary():
    tri = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    ev, et, ef = rwg_edges(tri)
    assert ev.tolist() == [[0, 2]]
    assert et.tolist() == [[0, 1]] and ef.tolist() == [[1, 3]]


def test_mie_optical_theorem_and_rayleigh():
    # energy balance of a lossless sphere: extinction == integrated scattering
    for ka_over_2pi in (0.3, 1.0, 2.0):
        a = ka_over_2pi
        th = np.linspace(0.0, np.pi, 4001)
        se = mie.pec_bistatic_eplane(a, 1.0, th)
        sh = mie.pec_bistatic_hplane(a, 1.0, th)
        # total scattered = (1/4pi) int sigma dOmega; average the two principal planes over phi
        integrand = 0.5 * (se + sh) * np.sin(th)
        trap = getattr(np, "trapezoid", None) or getattr(np, "trapz")
        sca = trap(integrand, th) * 2 * np.pi / (4 * np.pi)
        assert abs(sca - mie.pec_extinction(a, 1.0)) < 1e-5 * sca
    # Rayleigh limit of the PEC backscatter: sigma / (pi a^2) -> 9 (ka)^4
    a = 0.002
    ka = 2 * np.pi * a
    back = mie.pec_bistatic_eplane(a, 1.0, np.array([np.pi]))[0]
    assert abs(back / (np.pi * a * a) / (9 * ka ** 4) - 1.0) < 1e-3


def test_mom_sphere_rcs_matches_mie(sphere_small, dense_small):
    from synth import plane_wave_z
    k, p = plane_wave_z()
    b = sphere_small.rhs(k, p)
    x = np.linalg.solve(dense_small, b)[:, 0]
    th = np.deg2rad(np.arange(0, 181, 5))
    s = rcs.bistatic_theta_pol(sphere_small, x, th)
    sm = mie.pec_bistatic_eplane(0.3, 1.0, th)
    err_db = np.abs(rcs.db(s) - rcs.db(sm))
    assert err_db.max() < 0.5, err_db.max()


def test_galerkin_matrix_nearly_symmetric(dense_small):
    Z = dense_small
    asym = np.linalg.norm(Z - Z.T) / np.linalg.norm(Z)
    assert asym < 2e-3
    assert np.all(np.abs(np.diag(Z)) > 0)


def test_reciprocity_of_unmirrored_fill(sphere_small, dense_small):
    # Reaction reciprocity <E_A, J_B> = <E_B, J_A> holds for the physical operator;
    # the unmirrored quadrature breaks it only at the quadrature-error level.
    from synth import random_incidences
    k, p = random_incidences(2, seed=7)
    b = sphere_small.rhs(k, p)
    x = np.linalg.solve(dense_small, b)
    lhs, rhs = b[:, 0] @ x[:, 1], b[:, 1] @ x[:, 0]
    assert abs(lhs - rhs) < 2e-3 * abs(lhs)
