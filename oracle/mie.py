"""Mie series of a perfectly conducting sphere and of a homogeneous dielectric
sphere (textbook closed form, Bohren & Huffman 1983 §4.4; the conducting case
is the limit of the coefficients for an infinite refractive index).  Not in
arxiv 2307.03968; it pins the oracle's S-EFIE and V-EFIE fill, RHS and RCS.
Oracle — test infrastructure only.

A dielectric sphere (relative permittivity eps_r, mu = 1, refractive index
m = sqrt(eps_r)) has
  a_n = [m psi_n(mx) psi_n'(x) - psi_n(x) psi_n'(mx)] / [m psi_n(mx) xi_n'(x) - xi_n(x) psi_n'(mx)]
  b_n = [psi_n(mx) psi_n'(x) - m psi_n(x) psi_n'(mx)] / [psi_n(mx) xi_n'(x) - m xi_n(x) psi_n'(mx)].

With psi_n(x) = x j_n(x) and xi_n(x) = x h_n^(1)(x), a perfect conductor has
  a_n = psi_n'(x) / xi_n'(x),   b_n = psi_n(x) / xi_n(x),   x = k a,
  S1 = sum (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n),
  S2 = sum (2n+1)/(n(n+1)) (a_n tau_n + b_n pi_n),
with the angular functions pi_n, tau_n of cos(theta).  For incidence along +z
polarised along x, the bistatic RCS in the phi = 0 plane (E-plane, theta-pol)
is sigma = 4 pi |S2(theta)|^2 / k^2 and in the phi = 90 deg plane (H-plane,
phi-pol) 4 pi |S1(theta)|^2 / k^2.  The RCS does not depend on the time
convention.
"""

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def coefficients(x, nmax=None):
    if nmax is None:
        nmax = int(np.ceil(x + 4.05 * x ** (1.0 / 3.0) + 2))
    n = np.arange(1, nmax + 1)
    j, jd = spherical_jn(n, x), spherical_jn(n, x, derivative=True)
    y, yd = spherical_yn(n, x), spherical_yn(n, x, derivative=True)
    h, hd = j + 1j * y, jd + 1j * yd
    psi, dpsi = x * j, j + x * jd
    xi, dxi = x * h, h + x * hd
    return n, dpsi / dxi, psi / xi


def dielectric_coefficients(x, eps_r, nmax=None):
    if nmax is None:
        nmax = int(np.ceil(x + 4.05 * x ** (1.0 / 3.0) + 2))
    m = np.sqrt(eps_r)
    n = np.arange(1, nmax + 1)
    mx = m * x
    j, jd = spherical_jn(n, x), spherical_jn(n, x, derivative=True)
    y, yd = spherical_yn(n, x), spherical_yn(n, x, derivative=True)
    jm, jmd = spherical_jn(n, mx), spherical_jn(n, mx, derivative=True)
    h, hd = j + 1j * y, jd + 1j * yd
    psi, dpsi = x * j, j + x * jd
    xi, dxi = x * h, h + x * hd
    psim, dpsim = mx * jm, jm + mx * jmd
    a = (m * psim * dpsi - psi * dpsim) / (m * psim * dxi - xi * dpsim)
    b = (psim * dpsi - m * psi * dpsim) / (psim * dxi - m * xi * dpsim)
    return n, a, b


def amplitudes(x, theta, nmax=None, coeffs=None):
    n, a, b = coefficients(x, nmax) if coeffs is None else coeffs
    mu = np.cos(np.asarray(theta, dtype=np.float64))
    N = len(n)
    pi = np.zeros((N + 1,) + mu.shape)
    tau = np.zeros((N + 1,) + mu.shape)
    pi[1] = 1.0
    for k in range(2, N + 1):
        pi[k] = ((2 * k - 1) * mu * pi[k - 1] - k * pi[k - 2]) / (k - 1)
    for k in range(1, N + 1):
        tau[k] = k * mu * pi[k] - (k + 1) * pi[k - 1]
    c = ((2 * n + 1) / (n * (n + 1)))[:, None] if mu.ndim else (2 * n + 1) / (n * (n + 1))
    aa = a[:, None] if mu.ndim else a
    bb = b[:, None] if mu.ndim else b
    S1 = np.sum(c * (aa * pi[1:] + bb * tau[1:]), axis=0)
    S2 = np.sum(c * (aa * tau[1:] + bb * pi[1:]), axis=0)
    return S1, S2


def pec_bistatic_eplane(radius, wavelength, theta):
    """sigma_theta(theta), phi = 0, incidence +z x-polarised (m^2)."""
    k = 2 * np.pi / wavelength
    _, S2 = amplitudes(k * radius, theta)
    return 4 * np.pi * np.abs(S2) ** 2 / k ** 2


def pec_bistatic_hplane(radius, wavelength, theta):
    k = 2 * np.pi / wavelength
    S1, _ = amplitudes(k * radius, theta)
    return 4 * np.pi * np.abs(S1) ** 2 / k ** 2


def pec_extinction(radius, wavelength):
    """Optical theorem: sigma_ext = (4 pi / k^2) Re S(0)."""
    k = 2 * np.pi / wavelength
    S1, _ = amplitudes(k * radius, np.array([0.0]))
    return 4 * np.pi / k ** 2 * S1[0].real


def dielectric_bistatic_eplane(radius, wavelength, eps_r, theta):
    """sigma_theta(theta), phi = 0, incidence +z x-polarised (m^2)."""
    k = 2 * np.pi / wavelength
    x = k * radius
    _, S2 = amplitudes(x, theta, coeffs=dielectric_coefficients(x, eps_r))
    return 4 * np.pi * np.abs(S2) ** 2 / k ** 2


def dielectric_efficiencies(radius, wavelength, eps_r):
    """(Q_ext, Q_sca) of the lossless sphere; equal for a real eps_r."""
    x = 2 * np.pi / wavelength * radius
    n, a, b = dielectric_coefficients(x, eps_r)
    qext = 2 / x ** 2 * np.sum((2 * n + 1) * (a + b).real)
    qsca = 2 / x ** 2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    return qext, qsca
