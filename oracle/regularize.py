"""Regularization and parameter choice (oracle).

Projected problem (Sec. 3.3, eq. hybrid_problem; Algorithms 2 and 4):
C_l = U~ S~ V~^T, f~ = U~^T (beta_1 e_1) in R^{l+1}, filter factors
phi~_i(lambda) = s~_i^2 / (s~_i^2 + lambda^2), residual norm rho_l (eq.
rho_proj), solution norm eta_l (eq. eta_proj), GCV_l (eq. gcv_proj).

Full problem (Sec. 2.2 and 3.2; Algorithm 3): A = U S V^T, f^ = U^T f,
TSVD (eq. tsvd_solution), Tikhonov (eq. tikh_svd_solution), GCV (eq. gcv_svd).

Readings where the paper is silent or ambiguous:

* Projected SVD: Algorithm 2 asks for a thin SVD, but eq. rho_proj needs
  f~_{l+1}; the full U~ ((l+1) x (l+1)) is used so that f~ has l+1 entries.
* lambda grid: Algorithm 3 only says "log-grid", Algorithm 4 "argmin over
  lambda > 0".  Grid: lambda_t = s_1 * 10^t, t = linspace(-16, 0, 321) (0.05
  decade), where s_1 is the largest (Ritz) singular value; the choice is the
  grid argmin, smallest lambda among exactly equal values.
* GCV denominator on the projected problem: (l+1) - tr H_l, as printed in
  eq. gcv_proj (the full problem uses N - tr H, eq. gcv_svd).
* Evaluation of the filter terms: 1 - phi_i is evaluated as
  lambda^2 / (s_i^2 + lambda^2) and the denominators as
  (l+1) - sum phi~_i = 1 + sum (1 - phi~_i) and
  N - sum phi_i = (N - r) + sum (1 - phi_i).  These are the printed
  expressions rewritten exactly; they avoid the 0/0 that the literal form
  gives in floating point when lambda is far below every s_i.
* L-curve corner: x = ln rho, y = ln eta sampled on the same grid; signed
  curvature kappa = (x' y'' - x'' y') / (x'^2 + y'^2)^{3/2} with central
  differences in t over interior grid points; the corner is argmax kappa
  (positive at the corner when lambda increases along the curve).  Samples
  where the curve is stationary -- speed |(x', y')| below 1e-4 per decade of
  lambda, e.g. where rho and eta no longer change for lambda far below every
  s~_i -- have no meaningful curvature (rounding noise over a vanishing speed)
  and are not candidates; neither are samples where it is undefined.
* Ine-TSVD rank (the paper allows Picard plot, discrepancy or GCV; Sec. 5 uses
  GCV throughout): GCV_l(k) = (sum_{i=k+1}^{l} f~_i^2 + f~_{l+1}^2) / ((l+1) - k)^2,
  argmin over k = 1..r_l with r_l = #{s~_i > (l+1) eps s~_1}, smallest k on ties.
* Full-SVD numerical rank (Algorithm 3 uses r = rank(A)): r = #{s_i > N eps s_1};
  s_perp = |f|^2 - sum_{i<=r} f^_i^2; TSVD rank by
  GCV(k) = (sum_{k<i<=r} f^_i^2 + s_perp) / (N - k)^2 over k = 1..min(r, N-1)
  (k = N would leave a zero denominator).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

EPS = np.finfo(np.float64).eps
GRID_T_LO, GRID_T_HI, GRID_J = -16.0, 0.0, 321
# L-curve points whose speed |d(ln rho, ln eta)/dt| is below 1e-4 per decade are
# stationary: their discrete curvature is rounding noise over a vanishing speed.
LCURVE_MIN_SPEED2 = 1e-8


def lambda_grid(s1, J=GRID_J, t_lo=GRID_T_LO, t_hi=GRID_T_HI):
    """Log grid lambda_t = s1 * 10^t (Algorithm 3 input Lambda; reading above)."""
    return s1 * 10.0 ** np.linspace(t_lo, t_hi, J)


def grid_t(J=GRID_J, t_lo=GRID_T_LO, t_hi=GRID_T_HI):
    return np.linspace(t_lo, t_hi, J)


def _argmin_first(v):
    v = np.asarray(v)
    m = np.min(v)
    return int(np.flatnonzero(v == m)[0])


# ----------------------------------------------------------------------------
# projected problem
# ----------------------------------------------------------------------------

@dataclass
class ProjectedSVD:
    sigma: np.ndarray   # s~_1 >= ... >= s~_l
    ftil: np.ndarray    # f~ = U~^T (beta_1 e_1), length l+1
    V: np.ndarray       # V~ (l x l), columns v~_i
    U: np.ndarray       # U~ ((l+1) x (l+1))
    beta1: float

    @property
    def l(self):
        return self.sigma.shape[0]


def projected_svd(C, beta1) -> ProjectedSVD:
    """SVD of the bidiagonal C_l and f~ = U~^T (beta_1 e_1) (Alg. 2 step 2, Alg. 4 step 2)."""
    U, s, Vt = np.linalg.svd(C, full_matrices=True)
    ftil = U.T @ (beta1 * np.eye(C.shape[0])[:, 0])
    return ProjectedSVD(s, ftil, Vt.T, U, float(beta1))


def rho2_proj(ps: ProjectedSVD, lam):
    """rho_l^2(lambda) = sum_i (1 - phi~_i)^2 f~_i^2 + f~_{l+1}^2  (eq. rho_proj)."""
    l = ps.l
    out = np.empty(np.size(lam))
    for t, L in enumerate(np.atleast_1d(lam)):
        one_minus_ph = L * L / (ps.sigma ** 2 + L * L)
        out[t] = np.sum(one_minus_ph ** 2 * ps.ftil[:l] ** 2) + ps.ftil[l] ** 2
    return out


def eta2_proj(ps: ProjectedSVD, lam):
    """eta_l^2(lambda) = sum_i (phi~_i / s~_i)^2 f~_i^2  (eq. eta_proj)."""
    l = ps.l
    out = np.empty(np.size(lam))
    for t, L in enumerate(np.atleast_1d(lam)):
        ph = ps.sigma ** 2 / (ps.sigma ** 2 + L * L)
        with np.errstate(divide="ignore", invalid="ignore"):
            q = np.where(ps.sigma > 0, ph / ps.sigma, 0.0)
        out[t] = np.sum(q ** 2 * ps.ftil[:l] ** 2)
    return out


def gcv_proj(ps: ProjectedSVD, lam):
    """GCV_l(lambda) = rho_l^2 / ((l+1) - sum_i phi~_i)^2  (eq. gcv_proj)."""
    l = ps.l
    rho2 = rho2_proj(ps, lam)
    out = np.empty_like(rho2)
    for t, L in enumerate(np.atleast_1d(lam)):
        # (l+1) - sum_i phi~_i  =  1 + sum_i (1 - phi~_i)
        den = 1.0 + np.sum(L * L / (ps.sigma ** 2 + L * L))
        out[t] = rho2[t] / den ** 2
    return out


def lcurve_curvature(x, y, h):
    """Signed curvature of the sampled curve (x(t), y(t)), central differences.

    Returns kappa at interior samples 1..J-2 (array of length J-2).
    """
    x1 = (x[2:] - x[:-2]) / (2 * h)
    y1 = (y[2:] - y[:-2]) / (2 * h)
    x2 = (x[2:] - 2 * x[1:-1] + x[:-2]) / (h * h)
    y2 = (y[2:] - 2 * y[1:-1] + y[:-2]) / (h * h)
    return (x1 * y2 - x2 * y1) / (x1 * x1 + y1 * y1) ** 1.5


def choose_lambda_proj(ps: ProjectedSVD, rule="gcv", J=GRID_J):
    """lambda* on the grid by GCV (Alg. 4 step 5) or the L-curve corner (step 7).

    Returns (lambda*, index, grid, curve) where curve is GCV_l on the grid or
    the curvature at interior points.
    """
    t = grid_t(J)
    grid = lambda_grid(ps.sigma[0], J)
    if rule == "gcv":
        g = gcv_proj(ps, grid)
        i = _argmin_first(g)
        return grid[i], i, grid, g
    if rule == "lcurve":
        h = t[1] - t[0]
        with np.errstate(divide="ignore", invalid="ignore"):
            x = 0.5 * np.log(rho2_proj(ps, grid))
            y = 0.5 * np.log(eta2_proj(ps, grid))
            kap = lcurve_curvature(x, y, h)
            speed2 = ((x[2:] - x[:-2]) / (2 * h)) ** 2 + ((y[2:] - y[:-2]) / (2 * h)) ** 2
        kap = np.where(np.isfinite(kap) & (speed2 >= LCURVE_MIN_SPEED2), kap, -np.inf)
        m = np.max(kap)
        i = int(np.flatnonzero(kap == m)[0]) + 1
        return grid[i], i, grid, kap
    raise ValueError(rule)


def hkt_solve_proj(ps: ProjectedSVD, lam):
    """y_lambda solving (C^T C + lambda^2 I) y = C^T beta_1 e_1 (Alg. 4 step 9),
    in SVD form y = sum_i s~_i f~_i / (s~_i^2 + lambda^2) v~_i."""
    l = ps.l
    coef = ps.sigma * ps.ftil[:l] / (ps.sigma ** 2 + lam * lam)
    return ps.V @ coef


def numerical_rank_proj(ps: ProjectedSVD):
    if ps.l == 0 or ps.sigma[0] == 0.0:
        return 0
    return int(np.sum(ps.sigma > (ps.l + 1) * EPS * ps.sigma[0]))


def gcv_rank_proj(ps: ProjectedSVD):
    """GCV_l(k) for k = 1..r_l (reading above); returns (k*, curve)."""
    l = ps.l
    r = numerical_rank_proj(ps)
    f2 = ps.ftil ** 2
    curve = np.empty(r)
    for k in range(1, r + 1):
        curve[k - 1] = (np.sum(f2[k:l]) + f2[l]) / ((l + 1) - k) ** 2
    return _argmin_first(curve) + 1, curve


def tsvd_solve_proj(ps: ProjectedSVD, k):
    """y_k = sum_{i<=k} (f~_i / s~_i) v~_i  (Alg. 2 step 5)."""
    return ps.V[:, :k] @ (ps.ftil[:k] / ps.sigma[:k])


# ----------------------------------------------------------------------------
# methods on top of GKB
# ----------------------------------------------------------------------------

def hkt(g, rule="gcv", lam=None, J=GRID_J):
    """Hybrid Krylov-Tikhonov (Algorithm 4) on a finished GKB run ``g``.

    rule in {'gcv', 'lcurve', 'fixed'}; 'fixed' uses the given lambda; J grid
    points on the lambda grid.  Returns dict(coef = Z_l y_lambda, y, lam,
    index, ps, grid, curve).
    """
    ps = projected_svd(g.C(), g.beta1)
    if rule == "fixed":
        lam_s, idx, grid, curve = float(lam), -1, None, None
    else:
        lam_s, idx, grid, curve = choose_lambda_proj(ps, rule, J)
    y = hkt_solve_proj(ps, lam_s)
    coef = g.Z_l() @ y
    return dict(coef=coef, y=y, lam=float(lam_s), index=idx, ps=ps, grid=grid, curve=curve)


def ine_tsvd(g, rank=None):
    """Inexpensive TSVD (Algorithm 2): rank by GCV (reading) unless given."""
    ps = projected_svd(g.C(), g.beta1)
    if rank is None:
        k, curve = gcv_rank_proj(ps)
    else:
        k, curve = int(rank), None
    y = tsvd_solve_proj(ps, k)
    return dict(coef=g.Z_l() @ y, y=y, rank=k, ps=ps, curve=curve)


# ----------------------------------------------------------------------------
# full-SVD TSVD and Tikhonov (Sec. 2.2, Algorithm 3)
# ----------------------------------------------------------------------------

@dataclass
class FullSVD:
    U: np.ndarray
    sigma: np.ndarray
    V: np.ndarray
    fhat: np.ndarray
    r: int
    s_perp: float
    n: int


def full_svd(A, f, driver="gesdd") -> FullSVD:
    """Economy SVD of A, f^ = U^T f, s_perp = sum_{i>r} f^_i^2 (Alg. 3 steps 1-2).

    driver: the LAPACK routine, "gesdd" (divide and conquer, through NumPy) or
    "gesvd" (QR iteration, through SciPy): two backward-stable SVDs whose
    difference measures how much a result depends on rounding alone."""
    if driver == "gesdd":
        U, s, Vt = np.linalg.svd(A, full_matrices=False)
    elif driver == "gesvd":
        import scipy.linalg
        U, s, Vt = scipy.linalg.svd(A, full_matrices=False, lapack_driver="gesvd")
    else:
        raise ValueError(driver)
    n = A.shape[0]
    r = int(np.sum(s > n * EPS * s[0])) if s[0] > 0 else 0
    fhat = U.T @ f
    # s_perp: the energy of f outside the first r left singular vectors.  For the
    # square A the economy U is complete, so it is summed directly as in eq.
    # gcv_svd (Algorithm 3 writes |f|^2 - s_r, equal in exact arithmetic but
    # left with rounding noise when r = N).
    s_perp = float(np.sum(fhat[r:] ** 2))
    if U.shape[0] > U.shape[1]:
        s_perp += max(0.0, float(f @ f) - float(np.sum(fhat ** 2)))
    return FullSVD(U, s, Vt.T, fhat, r, s_perp, n)


def gcv_full(fs: FullSVD, lam):
    """GCV(lambda) = (sum_{i<=r}(1-phi_i)^2 f^_i^2 + s_perp) / (N - sum phi_i)^2 (eq. gcv_svd)."""
    s = fs.sigma[: fs.r]
    fh = fs.fhat[: fs.r]
    out = np.empty(np.size(lam))
    for t, L in enumerate(np.atleast_1d(lam)):
        one_minus_ph = L * L / (s ** 2 + L * L)
        # N - sum_{i<=r} phi_i  =  (N - r) + sum_{i<=r} (1 - phi_i)
        den = (fs.n - fs.r) + np.sum(one_minus_ph)
        out[t] = (np.sum(one_minus_ph ** 2 * fh ** 2) + fs.s_perp) / den ** 2
    return out


def tikhonov_full(A, f, rule="gcv", lam=None, fs=None):
    """Tikh-Rg (Algorithm 3): GCV grid argmin, then alpha_lambda (eq. tikh_svd_solution)."""
    fs = full_svd(A, f) if fs is None else fs
    if rule == "fixed":
        lam_s, idx, grid, g = float(lam), -1, None, None
    elif rule == "gcv":
        grid = lambda_grid(fs.sigma[0])
        g = gcv_full(fs, grid)
        idx = _argmin_first(g)
        lam_s = grid[idx]
    else:
        raise ValueError(rule)
    s = fs.sigma[: fs.r]
    ph = s ** 2 / (s ** 2 + lam_s ** 2)
    coef = fs.V[:, : fs.r] @ (ph / s * fs.fhat[: fs.r])
    return dict(coef=coef, lam=float(lam_s), index=idx, fs=fs, grid=grid, curve=g)


def tsvd_full(A, f, rank=None, fs=None):
    """Full TSVD (eq. tsvd_solution); rank by GCV (reading) unless given."""
    fs = full_svd(A, f) if fs is None else fs
    f2 = fs.fhat[: fs.r] ** 2
    if rank is None:
        kmax = min(fs.r, fs.n - 1)
        curve = np.array([(np.sum(f2[k:]) + fs.s_perp) / (fs.n - k) ** 2
                          for k in range(1, kmax + 1)])
        k = _argmin_first(curve) + 1
    else:
        k, curve = int(rank), None
    coef = fs.V[:, :k] @ (fs.fhat[:k] / fs.sigma[:k])
    return dict(coef=coef, rank=k, fs=fs, curve=curve)
