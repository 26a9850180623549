"""MQ basis, Helmholtz collocation entries and the Kansa matrix (oracle).

Sec. 2.1: u(X) ~ sum_j alpha_j phi(|X - X_j|) (eq. u_expansion); interior rows
apply L = Delta + k^2 (eqs. Lphi, H_entries); Dirichlet boundary rows are the
basis itself (R = B rows, since b(X) = 0 reduces eq. Robin to u = g);
A = [H; R] (eq. augmented_system).

Form of the basis.  The paper writes phi(r; eps) = sqrt(1 + eps^2 r^2)
(eq. MQ).  The workloads quote the shape parameter as c with
Phi(r) = sqrt(r^2 + c^2) = c * phi(r; 1/c).  ``form='c'`` (default) uses Phi;
``form='eps'`` uses phi with eps = 1/c, i.e. every entry divided by c.  Both
give the same reconstructed u when lambda is scaled by 1/c.

Closed form of the Laplacian (derived; the paper does not print it): with
s = r^2 + c^2, Phi' = r s^{-1/2}, Phi'' = c^2 s^{-3/2}, and in 3D
Delta Phi = Phi'' + (2/r) Phi' = (2 r^2 + 3 c^2) s^{-3/2}.
"""
from __future__ import annotations

import numpy as np


def phi(r, c):
    """Phi(r) = sqrt(r^2 + c^2)  (eq. MQ in c-form)."""
    r = np.asarray(r, dtype=np.float64)
    return np.sqrt(r * r + c * c)


def laplacian_phi(r, c):
    """Delta Phi = (2 r^2 + 3 c^2) / (r^2 + c^2)^{3/2} in R^3."""
    r = np.asarray(r, dtype=np.float64)
    s = r * r + c * c
    return (2.0 * r * r + 3.0 * c * c) / (s * np.sqrt(s))


def lphi(r, c, k):
    """L Phi = Delta Phi + k^2 Phi  (eqs. Lphi, H_entries)."""
    return laplacian_phi(r, c) + k * k * phi(r, c)


def distances(P, Q):
    """Euclidean distance matrix D_ij = |P_i - Q_j| (float64)."""
    P = np.asarray(P, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    diff = P[:, None, :] - Q[None, :, :]
    return np.sqrt(np.sum(diff * diff, axis=-1))


def assemble(X, n_interior, c, k, form="c"):
    """Kansa collocation matrix A = [H; R] (eq. augmented_system).

    Rows and columns follow the node order of X (interior nodes first, then
    boundary nodes); centres are the collocation points (Sec. 2.1).  Row i is
    L Phi(|X_i - X_j|) for i < n_interior and Phi(|X_i - X_j|) otherwise.  No row
    scaling is applied (the paper prescribes none).
    """
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    if not (0 <= n_interior <= n):
        raise ValueError("n_interior out of range")
    R = distances(X, X)
    A = np.empty((n, n))
    A[:n_interior] = lphi(R[:n_interior], c, k)
    A[n_interior:] = phi(R[n_interior:], c)
    if form == "eps":
        A /= c
    elif form != "c":
        raise ValueError(form)
    return A
