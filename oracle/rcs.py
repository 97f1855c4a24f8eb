"""Radar cross section from RWG current coefficients (the bistatic RCS of
arxiv 2307.03968 Figs. 2-4).  Oracle — test infrastructure only.

Far field of a surface current J (e^{jwt}):
  E_s(r) ~ -jk eta exp(-jkr)/(4 pi r) [F - r_hat (r_hat . F)],
  F(r_hat) = Int J(r') exp(+jk r_hat . r') dS'
so  sigma = 4 pi r^2 |E_s . p|^2 / |E_inc|^2 = (k eta)^2 / (4 pi) |p . F|^2
for a unit incident field and receive polarisation p (perpendicular to r_hat).
A volume polarisation current J = jw kappa D radiates the same way with
F = jw eps0 P, P = Int kappa (D/eps0) exp(+jk r_hat . r') dV', which gives
sigma = k^4 / (4 pi) |p . P|^2.  Each mesh class carries its factor as
``rcs_scale`` and its radiation vector as ``radiation``.
"""

import numpy as np


def bistatic_theta_pol(mesh, x, theta, phi=0.0):
    """sigma_theta (m^2) at observation angles theta (rad), fixed phi."""
    th = np.asarray(theta, dtype=np.float64)
    rhat = np.stack([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)], axis=1)
    that = np.stack([np.cos(th) * np.cos(phi), np.cos(th) * np.sin(phi), -np.sin(th)], axis=1)
    F = mesh.radiation(x, rhat)
    Ft = np.einsum('ij,ij->i', F, that)
    return mesh.rcs_scale * np.abs(Ft) ** 2


def monostatic(mesh, X, khat, phat):
    """Back-scattered sigma for each column of X (solution for incidence
    (khat[r], phat[r])), received in the incident polarisation."""
    out = np.empty(X.shape[1])
    for r in range(X.shape[1]):
        F = mesh.radiation(X[:, r], -khat[r:r + 1])[0]
        out[r] = mesh.rcs_scale * abs(np.dot(F, phat[r])) ** 2
    return out


def db(sigma, ref=1.0):
    return 10.0 * np.log10(np.asarray(sigma) / ref)
