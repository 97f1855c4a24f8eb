"""Plane-wave incidence parameters: propagation direction k_hat and unit
polarisation p_hat (p_hat perpendicular to k_hat), as float64 arrays (R, 3).

Only directions are generated here; evaluating the incident field on a mesh is
the solver's job (each side does it with its own code)."""

import numpy as np


def plane_wave_z():
    """Incidence along +z, x-polarised (one right-hand side)."""
    return np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]])


def monostatic_sweep(n_theta=181, phi=0.0):
    """Monostatic sweep theta = 0..180 deg (step 180/(n_theta-1)), given phi,
    theta-polarised.  The wave arrives from direction (theta, phi), so it
    propagates along -r_hat(theta, phi); the polarisation is theta_hat."""
    th = np.deg2rad(np.linspace(0.0, 180.0, n_theta))
    ph = np.full_like(th, phi)
    rhat = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    that = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], axis=1)
    return -rhat, that


def random_incidences(n, seed):
    """k_hat uniform on the sphere, p_hat uniform on the circle orthogonal to it."""
    rng = np.random.default_rng(seed)
    k = rng.normal(size=(n, 3))
    k /= np.linalg.norm(k, axis=1, keepdims=True)
    a = rng.normal(size=(n, 3))
    p = a - np.einsum('ij,ij->i', a, k)[:, None] * k
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    return k, p
