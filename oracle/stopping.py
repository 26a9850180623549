"""Oracle for the learned stop's inputs and labels: FP64, NumPy, slow and plain.

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the CPU
baseline of the benchmark, never by the product path.

* ``stop_features``: the 20 network inputs after j GKB steps, from their
  definitions: the singular values of the projected bidiagonal C_j (Sec. 3.1)
  and the least-squares residuals rho_i = min_y |C_i y - beta_1 e_1| of the
  projected problem after i steps (the LSQR residual, Sec. 3.4), each solved
  with a dense least-squares routine.
* ``error_table``: the max-norm error of the HKT reconstruction (Algorithm 4,
  eq. u_reconstruction) against a known field, for several l and lambda.
"""
from __future__ import annotations

import numpy as np

from . import evaluate as OE
from . import regularize as OR
from .lsqr import bidiag

NEG = -300.0  # stands for log10(0) and for unavailable entries


def stop_features(alpha, beta, j):
    """[log10 s~_1, log10(s~_i / s~_1) i = 2..10, log10(rho_i / beta_1) i = 1..10].

    alpha[i-1] = alpha_i, beta[i-1] = beta_i.  Singular values past j are NEG;
    residuals past j repeat the last one; a zero residual is NEG.
    """
    alpha = np.asarray(alpha, np.float64)
    beta = np.asarray(beta, np.float64)
    f = np.empty(20)
    C = bidiag(alpha, beta, j)
    s = np.linalg.svd(C, compute_uv=False)
    f[0] = np.log10(s[0])
    for i in range(1, 10):
        f[i] = np.log10(s[i] / s[0]) if i < j else NEG
    last = NEG
    for i in range(1, 11):
        if i <= j:
            Ci = bidiag(alpha, beta, i)
            rhs = np.zeros(i + 1)
            rhs[0] = beta[0]
            if beta[i] == 0.0:
                # beta_{i+1} = 0 (breakdown): the last row of C_i is zero and
                # the square lower bidiagonal block above it is nonsingular,
                # so the projected system is consistent and the residual is 0
                r = 0.0
            else:
                y = np.linalg.lstsq(Ci, rhs, rcond=None)[0]
                r = np.linalg.norm(Ci @ y - rhs)
            last = np.log10(r / beta[0]) if r > 0.0 else NEG
        f[9 + i] = last
    return f


def error_table(g, X, c, P, uref, ells, tgrid):
    """E[e, q] = max_t |u_t - uref_t| / max_t |uref_t| where u is the HKT
    reconstruction at P after ells[e] steps of the GKB run g with lambda =
    s~_1 10^tgrid[q]."""
    E = np.empty((len(ells), len(tgrid)))
    umax = np.max(np.abs(uref))
    for e, l in enumerate(ells):
        C = g.C()[: l + 1, :l]
        ps = OR.projected_svd(C, g.beta1)
        Z = g.Z_l()[:, :l]
        for q, t in enumerate(tgrid):
            y = OR.hkt_solve_proj(ps, ps.sigma[0] * 10.0 ** t)
            u = OE.reconstruct(Z @ y, X, P, c)
            E[e, q] = np.max(np.abs(u - uref)) / umax
    return E
