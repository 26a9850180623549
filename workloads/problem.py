"""Manufactured Helmholtz problems (eq. Helmholtz with Dirichlet data, Sec. 2.1).

* Plane wave u = sin(k d.X), |d| = 1: solves Delta u + k^2 u = 0 exactly, so the
  interior source is zero and the boundary data is u itself.
* Gaussian u = exp(-|X - X0|^2 / sigma) (Sec. 5, eq. exact_cube and the sphere and
  casing examples): its source is f = (4 rho^2/sigma^2 - 6/sigma + k^2) u with
  rho = |X - X0|.

The right-hand side is ordered like the node set: f = [f_I; g_B].
"""
from __future__ import annotations

import numpy as np

DIAG = np.array([1.0, 1.0, 1.0]) / np.sqrt(3.0)


def plane_wave(P: np.ndarray, k: float, d=DIAG) -> np.ndarray:
    d = np.asarray(d, dtype=np.float64)
    return np.sin(k * (P @ d))


def plane_wave_rhs(nodes, k: float, d=DIAG) -> np.ndarray:
    f = np.zeros(nodes.n)
    f[nodes.n_interior:] = plane_wave(nodes.X[nodes.n_interior:], k, d)
    return f


def gaussian(P: np.ndarray, sigma: float, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    q = P - np.asarray(center, dtype=np.float64)
    return np.exp(-np.sum(q * q, axis=1) / sigma)


def gaussian_source(P: np.ndarray, sigma: float, k: float, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    q = P - np.asarray(center, dtype=np.float64)
    rho2 = np.sum(q * q, axis=1)
    return (4.0 * rho2 / sigma ** 2 - 6.0 / sigma + k * k) * np.exp(-rho2 / sigma)


def gaussian_rhs(nodes, sigma: float, k: float, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    ni = nodes.n_interior
    return np.concatenate([gaussian_source(nodes.X[:ni], sigma, k, center),
                           gaussian(nodes.X[ni:], sigma, center)])


def instance_rhs(nodes) -> np.ndarray:
    """f for a node set whose params name its exact solution (see
    nodes.stop_instances): 'plane' (d) or 'gauss' (sigma, center)."""
    p = nodes.params
    if p.get("rhs", "plane") == "gauss":
        return gaussian_rhs(nodes, p["sigma"], p["k"], p["center"])
    return plane_wave_rhs(nodes, p["k"], p.get("d", DIAG))


def instance_field(nodes, P: np.ndarray) -> np.ndarray:
    """The exact solution of that instance at the points P."""
    p = nodes.params
    if p.get("rhs", "plane") == "gauss":
        return gaussian(P, p["sigma"], p["center"])
    return plane_wave(P, p["k"], p.get("d", DIAG))
