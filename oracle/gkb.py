"""Golub-Kahan bidiagonalization, Lanczos form (Algorithm 1, Sec. 3.1) -- oracle.

Notation follows the paper: w_j (left basis, W), z_j (right basis, Z), alpha_j
on the diagonal and beta_{j+1} on the subdiagonal of the lower-bidiagonal
C_l in R^{(l+1) x l}; beta_1 = |f|, w_1 = f / beta_1, z_0 = 0.

Readings where Algorithm 1 is ambiguous or silent:

* Reorthogonalization placement.  Algorithm 1 lists an optional
  reorthogonalization of w_{j+1} and z_j after they are normalised and never
  renormalises.  Here the unnormalised r is reorthogonalized against
  z_1..z_{j-1} before alpha_j = |r|, and p against w_1..w_j before
  beta_{j+1} = |p|, so that (alpha_j, beta_{j+1}) are the norms of the vectors
  actually stored.  Reorthogonalization is always full.
* Reorthogonalization scheme.  ``reorth='mgs2'`` (default): modified
  Gram-Schmidt applied twice.  ``reorth='cgs2'``: classical Gram-Schmidt
  applied twice ("twice is enough", Giraud et al. 2005).  Both give the same
  vectors in exact arithmetic.
* Breakdown threshold (the paper only says the process halts when some
  alpha_j or beta_{j+1} vanishes).  tau = 64 * N * eps_mach * c_hat, where c_hat
  is a running lower estimate of |A|_2: the maximum over completed columns i of
  sqrt(alpha_i^2 + beta_{i+1}^2), and alpha_j itself while alpha_j is tested.
  If alpha_j <= tau the run stops with l_done = j - 1.  If beta_{j+1} <= tau the
  run stops with l_done = j, and beta_{j+1} and w_{j+1} are set to exactly zero
  (an invariant subspace was found).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

EPS = np.finfo(np.float64).eps
BREAKDOWN_FACTOR = 64.0


@dataclass
class GKBResult:
    W: np.ndarray        # N x (steps+1); columns 0..l_done valid
    Z: np.ndarray        # N x steps;     columns 0..l_done-1 valid
    alpha: np.ndarray    # alpha[j-1] = alpha_j
    beta: np.ndarray     # beta[j-1]  = beta_j  (beta[0] = beta_1 = |f|)
    steps_done: int
    breakdown: int       # 0 none, 1 alpha breakdown, 2 beta breakdown
    c_hat: float

    @property
    def beta1(self) -> float:
        return float(self.beta[0])

    def C(self) -> np.ndarray:
        """Lower bidiagonal C_l ((l+1) x l): diag alpha_1..alpha_l, subdiag beta_2..beta_{l+1}."""
        l = self.steps_done
        C = np.zeros((l + 1, l))
        for j in range(l):
            C[j, j] = self.alpha[j]
            C[j + 1, j] = self.beta[j + 1]
        return C

    def W_l1(self) -> np.ndarray:
        return self.W[:, : self.steps_done + 1]

    def Z_l(self) -> np.ndarray:
        return self.Z[:, : self.steps_done]


def _reorth(v, Q, scheme):
    """Remove from v its components along the orthonormal columns of Q, twice."""
    for _ in range(2):
        if scheme == "mgs2":
            for i in range(Q.shape[1]):
                q = Q[:, i]
                v = v - (q @ v) * q
        elif scheme == "cgs2":
            if Q.shape[1]:
                v = v - Q @ (Q.T @ v)
        else:
            raise ValueError(scheme)
    return v


def gkb(matvec, rmatvec, f, steps, n=None, reorth="mgs2") -> GKBResult:
    """Run l = ``steps`` steps of Algorithm 1.

    ``matvec(x)`` returns A x and ``rmatvec(y)`` returns A^T y; a dense array
    may be passed as ``matvec`` instead (then ``rmatvec`` may be None).
    """
    if isinstance(matvec, np.ndarray):
        A = matvec
        matvec, rmatvec = (lambda x: A @ x), (lambda y: A.T @ y)
    f = np.asarray(f, dtype=np.float64)
    N = f.shape[0] if n is None else n
    W = np.zeros((N, steps + 1))
    Z = np.zeros((N, steps))
    alpha = np.zeros(steps)
    beta = np.zeros(steps + 1)
    beta1 = float(np.linalg.norm(f))
    beta[0] = beta1
    if beta1 == 0.0:
        return GKBResult(W, Z, alpha, beta, 0, 1, 0.0)
    W[:, 0] = f / beta1
    c_hat = 0.0
    z_prev = np.zeros(N)
    for j in range(1, steps + 1):
        # r = A^T w_j - beta_j z_{j-1}
        r = rmatvec(W[:, j - 1]) - beta[j - 1] * z_prev
        r = _reorth(r, Z[:, : j - 1], reorth)
        a = float(np.linalg.norm(r))
        tau = BREAKDOWN_FACTOR * N * EPS * max(c_hat, a)
        if a <= tau:
            return GKBResult(W, Z, alpha, beta, j - 1, 1, c_hat)
        alpha[j - 1] = a
        Z[:, j - 1] = r / a
        # p = A z_j - alpha_j w_j
        p = matvec(Z[:, j - 1]) - a * W[:, j - 1]
        p = _reorth(p, W[:, :j], reorth)
        b = float(np.linalg.norm(p))
        c_hat = max(c_hat, float(np.hypot(a, b)))
        tau = BREAKDOWN_FACTOR * N * EPS * c_hat
        if b <= tau:
            beta[j] = 0.0
            return GKBResult(W, Z, alpha, beta, j, 2, c_hat)
        beta[j] = b
        W[:, j] = p / b
        z_prev = Z[:, j - 1]
    return GKBResult(W, Z, alpha, beta, steps, 0, c_hat)
