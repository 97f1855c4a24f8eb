"""Pins of the oracle's multi-level power series (arxiv 2307.03968 §IV).

- leaf level: the block implementation equals sum_k (-U)^k D^{-1} b with dense
  powers of U = D^{-1} M_1 (brute force), and obeys the Neumann truncation
  identity x* - x_K = (-U)^{K+1} x*;
- K -> infinity: nested (eq. 19) and flat forms both reach the closed form
  A_m^{-1} b of the telescoped eqs. 12-19 (on an operator damped so the series
  converges);
- special cases: a single leaf gives the exact solve, zero coupling gives
  D^{-1} b, a random diagonal alpha (eqs. 9-12) changes nothing;
- reciprocity: every form is a symmetric operator applied to b;
- one refinement step squares the truncation factor;
- at finite K on an operator with far blocks on three levels: the nested form
  (eq. 19) at m = 1, 2, 3 levels, plain and refined, and the flat form equal the
  same operators written as dense matrix products (P_0 = D^{-1},
  P_m = sum_{k<=K} (-P_{m-1} M_m)^k P_{m-1}), with explicit matrix powers.
"""

import copy

import numpy as np
import pytest

from oracle import series
from oracle.hmatrix import HMatrix


@pytest.fixture(scope="module")
def hm2(sphere_small):
    return HMatrix(sphere_small, leaf_size=32, arity=2, adm=1.0, aca_tol=1e-4)


def damped(H, s):
    """A copy of H with every off-diagonal block scaled by s."""
    G = copy.copy(H)
    G.near = [(a, b, c, d, s * B) for (a, b, c, d, B) in H.near]
    G.far = {lev: [(a, b, c, d, s * U, V) for (a, b, c, d, U, V) in lst] for lev, lst in H.far.items()}
    return G


def dense_parts(H):
    I = np.eye(H.N, dtype=np.complex128)
    D = H.apply_D(I)
    M = {lev: H.apply_M(lev, I) for lev in range(1, H.n_levels + 1)}
    return D, M


@pytest.fixture(scope="module")
def rhs2(sphere_small):
    from synth import random_incidences
    k, p = random_incidences(3, seed=11)
    return sphere_small.rhs(k, p)


def test_leaf_series_equals_dense_powers(hm2, rhs2):
    H = hm2
    D, M = dense_parts(H)
    U = np.linalg.solve(D, M[1])
    bt = H.to_tree(rhs2)
    y = np.linalg.solve(D, bt)
    for K in (0, 1, 2, 3):
        ref = sum(np.linalg.matrix_power(-U, k) @ y for k in range(K + 1))
        got = H.to_tree(series.solve(H, rhs2, K=K, levels=1))
        assert np.linalg.norm(got - ref) < 1e-11 * np.linalg.norm(ref), K


def test_neumann_truncation_identity(hm2, rhs2):
    H = hm2
    D, M = dense_parts(H)
    A1 = D + M[1]
    U = np.linalg.solve(D, M[1])
    bt = H.to_tree(rhs2)
    xs = np.linalg.solve(A1, bt)
    for K in (1, 2, 3):
        xk = H.to_tree(series.solve(H, rhs2, K=K, levels=1))
        pred = np.linalg.matrix_power(-U, K + 1) @ xs
        assert np.linalg.norm((xs - xk) - pred) < 1e-9 * np.linalg.norm(pred)


@pytest.mark.parametrize("nested_form", [True, False])
def test_series_converges_to_closed_form(hm2, rhs2, nested_form):
    H = damped(hm2, 0.02)          # spectral radius of D^{-1}(A_2 - D) ~ 0.05
    D, M = dense_parts(H)
    bt = H.to_tree(rhs2)
    assert H.n_levels == 2
    for m in (1, 2):
        Am = D + sum(M[l] for l in range(1, m + 1))
        xs = np.linalg.solve(Am, bt)
        x = H.to_tree(series.solve(H, rhs2, K=12, levels=m, nested_form=nested_form))
        assert np.linalg.norm(x - xs) < 1e-11 * np.linalg.norm(xs)


def test_nested_equals_flat_at_leaf_level(hm2, rhs2):
    a = series.solve(hm2, rhs2, K=2, levels=1, nested_form=True)
    b = series.solve(hm2, rhs2, K=2, levels=1, nested_form=False)
    assert np.array_equal(a, b)


def test_nested_level_equation(hm2, rhs2):
    """P_2 r solves (I + T_2) x = y up to the truncation term (-T_2)^{K+1} y,
    with y = P_1 r and T_2 = P_1 M_2 (eqs. 15-18 at finite K)."""
    H = hm2
    D, M = dense_parts(H)
    K = 2
    Dinv = np.linalg.inv(D)
    U1 = Dinv @ M[1]
    P1 = sum(np.linalg.matrix_power(-U1, k) for k in range(K + 1)) @ Dinv
    T2 = P1 @ M[2]
    bt = H.to_tree(rhs2)
    y = P1 @ bt
    x = H.to_tree(series.solve(H, rhs2, K=K, levels=2))
    lhs = x + T2 @ x
    rhs = y - np.linalg.matrix_power(-T2, K + 1) @ y
    assert np.linalg.norm(lhs - rhs) < 1e-9 * np.linalg.norm(rhs)


def test_alpha_scaling_cancels(hm2, rhs2):
    rng = np.random.default_rng(5)
    alpha = rng.uniform(0.5, 2.0, hm2.N) * np.exp(1j * rng.uniform(0, 2 * np.pi, hm2.N))
    bt = hm2.to_tree(rhs2)
    for m in (1, 2):
        a = series.nested(hm2, bt, 2, m)
        b = series.nested(hm2, bt, 2, m, alpha=alpha)
        assert np.linalg.norm(a - b) < 1e-11 * np.linalg.norm(a)


def test_single_leaf_is_exact_solve(sphere_tiny):
    H = HMatrix(sphere_tiny, leaf_size=sphere_tiny.ne, arity=8)
    assert H.depth == 0 and not H.near and not H.far
    from synth import plane_wave_z
    b = sphere_tiny.rhs(*plane_wave_z())
    Z = sphere_tiny.dense()
    iu = np.triu_indices(H.N, 1)
    Zt = Z[np.ix_(H.perm, H.perm)]
    Zt[(iu[1], iu[0])] = Zt[iu]
    ref = H.from_tree(np.linalg.solve(Zt, H.to_tree(b)))
    for K in (0, 2):
        x = series.solve(H, b, K=K, levels=-1, refine=True)
        assert np.linalg.norm(x - ref) < 1e-12 * np.linalg.norm(ref)


def test_zero_coupling_gives_leaf_solve(hm2, rhs2):
    H = damped(hm2, 0.0)
    bt = H.to_tree(rhs2)
    ref = H.from_tree(H.solve_D(bt))
    for m in (1, 2):
        x = series.solve(H, rhs2, K=2, levels=m)
        assert np.linalg.norm(x - ref) < 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("levels,nested_form", [(1, True), (2, True), (2, False)])
def test_reciprocity_of_series(hm2, rhs2, levels, nested_form):
    x = series.solve(hm2, rhs2, K=2, levels=levels, nested_form=nested_form, refine=True)
    for a, b in ((0, 1), (0, 2), (1, 2)):
        lhs, rhs = rhs2[:, a] @ x[:, b], rhs2[:, b] @ x[:, a]
        assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_refinement_squares_truncation(hm2, rhs2):
    H = damped(hm2, 0.2)
    D, M = dense_parts(H)
    U = np.linalg.solve(D, M[1])
    bt = H.to_tree(rhs2)
    xs = np.linalg.solve(D + M[1], bt)
    K = 2
    x = H.to_tree(series.solve(H, rhs2, K=K, levels=1, refine=True))
    pred = np.linalg.matrix_power(-U, 2 * (K + 1)) @ xs
    assert np.linalg.norm((xs - x) - pred) < 1e-9 * np.linalg.norm(pred)


@pytest.fixture(scope="module")
def hm3(sphere_small):
    """The 1,920-unknown sphere on a binary tree with leaves of 16: far blocks on three
    levels (about 2,300, 640 and 4 of them)."""
    H = HMatrix(sphere_small, leaf_size=16, arity=2, adm=1.0, aca_tol=1e-4)
    assert H.n_levels == 3 and all(len(H.far.get(lev, [])) > 0 for lev in (1, 2, 3))
    return H


@pytest.fixture(scope="module")
def dense3(hm3):
    """D, M_1..M_3 and, for K = 1 and 2, the dense P_1 and P_2 of eq. 19."""
    D, M = dense_parts(hm3)
    Dinv = np.linalg.inv(D)
    P = {}
    for K in (1, 2):
        Pm = Dinv
        for lev in (1, 2):
            T = Pm @ M[lev]
            S = sum(np.linalg.matrix_power(-T, k) for k in range(K + 1))
            Pm = S @ Pm
            P[K, lev] = Pm
        P[K, 0] = Dinv
    return D, M, P


def dense_apply_P(dense, K, m, v):
    """P_m v from the dense matrices: P_1, P_2 as formed above; P_3 v = S_K(T_3)(P_2 v)
    with T_3 = P_2 M_3, as the explicit sum of matrix powers applied to P_2 v."""
    D, M, P = dense
    if m <= 2:
        return P[K, m] @ v
    T = P[K, 2] @ M[3]
    y = P[K, 2] @ v
    return sum(np.linalg.matrix_power(-T, k) @ y for k in range(K + 1))


@pytest.mark.parametrize("K", [1, 2])
@pytest.mark.parametrize("m", [1, 2, 3])
def test_nested_series_equals_dense_products_on_three_levels(hm3, dense3, rhs2, K, m):
    bt = hm3.to_tree(rhs2)
    ref = dense_apply_P(dense3, K, m, bt)
    got = hm3.to_tree(series.solve(hm3, rhs2, K=K, levels=m))
    assert np.linalg.norm(got - ref) < 1e-10 * np.linalg.norm(ref)


def test_refined_nested_series_equals_dense_products_on_three_levels(hm3, dense3, rhs2):
    D, M, _ = dense3
    A = D + M[1] + M[2] + M[3]
    bt = hm3.to_tree(rhs2)
    x1 = dense_apply_P(dense3, 2, 3, bt)
    ref = x1 + dense_apply_P(dense3, 2, 3, bt - A @ x1)
    got = hm3.to_tree(series.solve(hm3, rhs2, K=2, levels=-1, refine=True))
    assert np.linalg.norm(got - ref) < 1e-10 * np.linalg.norm(ref)


def test_flat_series_equals_dense_powers_on_three_levels(hm3, dense3, rhs2):
    D, M, P = dense3
    U = P[1, 0] @ (M[1] + M[2] + M[3])
    y = P[1, 0] @ hm3.to_tree(rhs2)
    ref = sum(np.linalg.matrix_power(-U, k) @ y for k in range(3))
    got = hm3.to_tree(series.solve(hm3, rhs2, K=2, levels=3, nested_form=False))
    assert np.linalg.norm(got - ref) < 1e-10 * np.linalg.norm(ref)


def test_nested_and_flat_differ_beyond_the_leaf_level(hm3, rhs2):
    """The two forms agree at m = 1 and differ at finite K for m > 1 (the nested form
    re-applies the inner series inside every outer term), so the pins above tell them apart."""
    a = series.solve(hm3, rhs2, K=2, levels=3, nested_form=True)
    b = series.solve(hm3, rhs2, K=2, levels=3, nested_form=False)
    assert np.linalg.norm(a - b) > 1e-6 * np.linalg.norm(a)
