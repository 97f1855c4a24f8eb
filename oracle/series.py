"""Multi-level power-series solution (arxiv 2307.03968 §IV, eqs. 8-22).

Oracle — test infrastructure only.  Vectors are (N, R) complex128 in tree
order unless stated otherwise.

Notation (readings of the paper where it is silent or ambiguous):
  D        block diagonal of the leaf self blocks of Z_N: the "[Z~_N]^{-1}" of
           eq. 12 is read as D^{-1} (the near field is made block diagonal on
           the leaf partition; the scaling alpha of eqs. 9-11 cancels for any
           alpha that is block diagonal on that partition, see ``alpha`` below);
  M_1      non-self near blocks + far blocks at the leaf level (the leaf-level
           operator; the solve "starts from the leaf level", §IV and abstract);
  M_l      far blocks l-1 levels above the leaves (eq. 8's Z_Fl, counted from
           the leaf);
  A_m      D + M_1 + ... + M_m, the H-Matrix truncated at m levels;
  S_K(T)y  sum_{k=0..K} (-T)^k y, evaluated as x_0 = y, x_j = y - T x_{j-1};
           this is the power series of (I + T)^{-1} (eq. 20-22, ref. [18,19]),
           truncated after K applications of T ("two fixed iterations": K = 2).

Nested form, literal eqs. 13-19:
  P_0(r) = D^{-1} r
  P_m(r) = S_K(T_m)(P_{m-1}(r)),   T_m(z) = P_{m-1}(M_m z)
so that P_1 = (I + U_1)^{-1} D^{-1} with U_1 = D^{-1} M_1, and for exact inner
inverses P_m = (I + V_m)^{-1} P_{m-1} = A_m^{-1} (the product of eq. 19
telescopes).  Flat form: x = S_K(D^{-1}(A_m - D))(D^{-1} r); identical to the
nested form for m = 1 and with the same K -> infinity limit A_m^{-1} r.
"""

import numpy as np


def nested(H, r, K, m, alpha=None):
    """P_m(r) of the nested recursion (eq. 19).  ``alpha`` (length-N diagonal
    scaling in tree order, eqs. 9-12): if given, the leaf solve uses
    Z~_N = alpha Z_N and every level operator is alpha M_l, with r -> alpha r."""
    if alpha is not None:
        a = alpha[:, None]

        def P0(v):
            return H.solve_D(v / a)   # (alpha D)^{-1} v = D^{-1} alpha^{-1} v

        def Mop(level, v):
            return a * H.apply_M(level, v)
        r = a * r
    else:
        P0 = H.solve_D

        def Mop(level, v):
            return H.apply_M(level, v)

    def P(level, v):
        if level == 0:
            return P0(v)
        y = P(level - 1, v)
        x = y
        for _ in range(K):
            x = y - P(level - 1, Mop(level, x))
        return x

    return P(m, r)


def flat(H, r, K, m):
    """x = S_K(D^{-1}(A_m - D))(D^{-1} r): one pass over all m levels per term."""
    y = H.solve_D(r)
    x = y
    for _ in range(K):
        z = np.zeros_like(x)
        for lev in range(1, m + 1):
            z += H.apply_M(lev, x)
        x = y - H.solve_D(z)
    return x


def solve(H, b, K=2, levels=1, nested_form=True, refine=False):
    """The power-series solution in the ORIGINAL unknown order.

    b: (N,) or (N, R).  levels: 1 = leaf level only (the paper's runs), m > 1 =
    m levels from the leaf, -1 = all levels.  refine: one refinement step
    x += P_m(b - A_m x) with the same K and levels."""
    vec = b.ndim == 1
    bt = H.to_tree(b.reshape(len(b), -1).astype(np.complex128))
    m = H.n_levels if levels is None or levels < 0 else min(levels, H.n_levels)
    m = max(m, 1)

    def P(v):
        return nested(H, v, K, m) if nested_form else flat(H, v, K, m)

    x = P(bt)
    if refine:
        x = x + P(bt - H.apply(x, m))
    out = H.from_tree(x)
    return out[:, 0] if vec else out
