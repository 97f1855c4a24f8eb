"""Restarted GMRES on the oracle's H-Matrix product: the iterative solver the paper
compares its power series with (arxiv 2307.03968 §IV, GMRES to a relative residual
of 1e-6 on the full H-Matrix).  Oracle — test infrastructure only.

Plain unpreconditioned GMRES(restart) with modified Gram-Schmidt Arnoldi and
Givens rotations, written out (no library solver), in complex128; the
right-hand side and iterate are in tree order like the H-Matrix operator."""

import numpy as np


def gmres(apply, b, tol=1e-6, restart=100, maxiter=5000):
    """Solve A x = b for the linear map `apply` (vector -> vector).  Returns
    (x, iterations, relative residual history); stops at |b - A x| <= tol |b|."""
    b = np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    hist = []
    it = 0
    if nb == 0.0:
        return x, 0, [0.0]
    while it < maxiter:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        hist.append(beta / nb)
        if beta <= tol * nb:
            break
        m = min(restart, maxiter - it)
        Q = np.zeros((m + 1, b.size), dtype=np.complex128)
        Hs = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        Q[0] = r / beta
        k_used = 0
        for k in range(m):
            w = apply(Q[k])
            for i in range(k + 1):               # modified Gram-Schmidt
                Hs[i, k] = np.vdot(Q[i], w)
                w = w - Hs[i, k] * Q[i]
            Hs[k + 1, k] = np.linalg.norm(w)
            if Hs[k + 1, k] != 0:
                Q[k + 1] = w / Hs[k + 1, k]
            # rotations G_i = [[conj(c_i), conj(s_i)], [-s_i, c_i]] (unitary, |c|^2 + |s|^2 = 1)
            for i in range(k):                   # previous rotations
                t = np.conj(cs[i]) * Hs[i, k] + np.conj(sn[i]) * Hs[i + 1, k]
                Hs[i + 1, k] = -sn[i] * Hs[i, k] + cs[i] * Hs[i + 1, k]
                Hs[i, k] = t
            a, c = Hs[k, k], Hs[k + 1, k]        # new rotation zeroing H[k+1, k]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            cs[k], sn[k] = (a / den, c / den) if den > 0 else (1.0, 0.0)
            Hs[k, k] = den
            Hs[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = np.conj(cs[k]) * g[k]
            it += 1
            k_used = k + 1
            hist.append(abs(g[k + 1]) / nb)
            if abs(g[k + 1]) <= tol * nb:
                break
        y = np.linalg.solve(np.triu(Hs[:k_used, :k_used]), g[:k_used])
        x = x + Q[:k_used].T @ y
        if hist[-1] <= tol:
            r = b - apply(x)
            if np.linalg.norm(r) <= tol * nb * 1.01:
                break
    return x, it, hist
