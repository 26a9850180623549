"""Oracle for LSQR as iterative regularization (Sec. 3.4): FP64, NumPy, plain.

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the CPU
baseline of the benchmark, never by the product path.

After k GKB steps the LSQR iterate is x_k = Z_k y_k with y_k the least-squares
solution of the projected problem C_k y = beta_1 e_1 (the Krylov subspace of
the first k right basis vectors).  Early stopping picks k from the sequence
(rho_k, eta_k) = (|A x_k - f|, |x_k|) = (|C_k y_k - beta_1 e_1|, |y_k|):

* 'lcurve': the corner of the discrete L-curve (ln rho_k, ln eta_k), taken as
  the maximum signed curvature by central differences, the sequence ordered by
  decreasing k (more regularization along the curve, as with growing lambda);
  points whose speed is below the stationarity floor are not candidates;
* 'gcv': argmin_k rho_k^2 / ((l + 1) - k)^2, the projected GCV with the
  k-dimensional Krylov filter's trace k (readings: the paper names the L-curve
  and GCV variants without formulas).
"""
from __future__ import annotations

import numpy as np

from .regularize import LCURVE_MIN_SPEED2, lcurve_curvature


def bidiag(alpha, beta, k):
    """Lower bidiagonal C_k ((k+1) x k): alpha_1..alpha_k on the diagonal,
    beta_2..beta_{k+1} below it (Algorithm 1)."""
    C = np.zeros((k + 1, k))
    for m in range(k):
        C[m, m] = alpha[m]
        C[m + 1, m] = beta[m + 1]
    return C


def lsqr_sequence(alpha, beta, l):
    """rho[k-1], eta[k-1], and y_k (list) for k = 1..l, each by dense least squares."""
    rho = np.empty(l)
    eta = np.empty(l)
    ys = []
    for k in range(1, l + 1):
        C = bidiag(alpha, beta, k)
        rhs = np.zeros(k + 1)
        rhs[0] = beta[0]
        y = np.linalg.lstsq(C, rhs, rcond=None)[0]
        rho[k - 1] = 0.0 if beta[k] == 0.0 else np.linalg.norm(C @ y - rhs)
        eta[k - 1] = np.linalg.norm(y)
        ys.append(y)
    return rho, eta, ys


def choose_k(rho, eta, l, rule):
    """Stopping index k (1-based) and the rule's curve over k = 1..l."""
    if rule == "gcv":
        k = np.arange(1, l + 1)
        g = rho ** 2 / ((l + 1) - k) ** 2.0
        i = int(np.flatnonzero(g == np.min(g))[0])
        return i + 1, g
    if rule == "lcurve":
        if l < 3:
            return l, np.full(l, -np.inf)
        with np.errstate(divide="ignore", invalid="ignore"):
            x = np.log(rho[::-1])
            y = np.log(eta[::-1])
            kap = lcurve_curvature(x, y, 1.0)
            speed2 = ((x[2:] - x[:-2]) / 2.0) ** 2 + ((y[2:] - y[:-2]) / 2.0) ** 2
        kap = np.where(np.isfinite(kap) & (speed2 >= LCURVE_MIN_SPEED2), kap, -np.inf)
        curve = np.full(l, -np.inf)
        curve[1:-1] = kap[::-1]          # curve[k-1] for k = 2..l-1
        m = np.max(curve)
        if not np.isfinite(m):
            return l, curve
        i = int(np.flatnonzero(curve == m)[0])
        return i + 1, curve
    raise ValueError(rule)


def lsqr_solve(g, rule="lcurve", k=None):
    """Early-stopped LSQR on a finished GKB run g: dict(coef, k, rho, eta, curve)."""
    l = g.steps_done
    rho, eta, ys = lsqr_sequence(g.alpha, g.beta, l)
    if rule == "fixed":
        kk, curve = int(k), None
    else:
        kk, curve = choose_k(rho, eta, l, rule)
    coef = g.Z[:, :kk] @ ys[kk - 1]
    return {"coef": coef, "k": kk, "rho": rho, "eta": eta, "curve": curve, "y": ys[kk - 1]}
