"""Reconstruction and error (oracle).

u_a(X) = sum_j alpha_j Phi(|X - X_j|)  (eqs. u_expansion, u_reconstruction:
the basis itself, not L Phi, at evaluation points), and
Re = |u - u_a|_inf / |u|_inf  (eq. rel_error).
"""
from __future__ import annotations

import numpy as np

from .mq import distances, phi


def reconstruct(coef, X, P, c, form="c", block=512):
    """u_a at the rows of P from coefficients on the centres X."""
    P = np.asarray(P, dtype=np.float64)
    out = np.empty(P.shape[0])
    for s in range(0, P.shape[0], block):
        B = phi(distances(P[s:s + block], X), c)
        if form == "eps":
            B /= c
        out[s:s + block] = B @ coef
    return out


def rel_error(u, ua):
    """Re = max |u - u_a| / max |u|  (eq. rel_error)."""
    return float(np.max(np.abs(u - ua)) / np.max(np.abs(u)))


def rms_error(u, ua):
    return float(np.sqrt(np.mean((u - ua) ** 2)))
