"""Oracle pins: projected SVD, GCV, L-curve, Ine-TSVD, HKT, full TSVD/Tikhonov."""
import math

import numpy as np
import pytest

import pins
from oracle import gkb as G
from oracle import mq
from oracle import regularize as R


def _gkb(n=120, ni=80, l=30, c=0.25, k=3.0, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (n, 3))
    A = mq.assemble(X, ni, c, k)
    f = rng.normal(size=n)
    return A, f, G.gkb(A, None, f, l)


def test_projected_svd_pins():
    _, _, g = _gkb()
    ps = R.projected_svd(g.C(), g.beta1)
    pins.pin_projected_svd(ps, g.C(), g.beta1)


def test_gcv_matches_dense_hat_matrix():
    _, _, g = _gkb(l=20)
    C = g.C()
    ps = R.projected_svd(C, g.beta1)
    for t in (-8, -4, -2, -1, 0):
        lam = ps.sigma[0] * 10.0 ** t
        ref = pins.gcv_dense(C, g.beta1, lam)
        assert R.gcv_proj(ps, lam)[0] == pytest.approx(ref, rel=1e-9)


def test_gcv_limits():
    _, _, g = _gkb(l=25)
    ps = R.projected_svd(g.C(), g.beta1)
    l = ps.l
    big = R.gcv_proj(ps, ps.sigma[0] * 1e9)[0]
    assert big == pytest.approx(g.beta1 ** 2 / (l + 1) ** 2, rel=1e-12)
    small = R.gcv_proj(ps, ps.sigma[-1] * 1e-9)[0]
    assert small == pytest.approx(ps.ftil[l] ** 2, rel=1e-6)


def test_gcv_grid_argmin_brute_force():
    _, _, g = _gkb(l=25, seed=3)
    C = g.C()
    ps = R.projected_svd(C, g.beta1)
    lam, idx, grid, curve = R.choose_lambda_proj(ps, "gcv")
    dense = np.array([pins.gcv_dense(C, g.beta1, L) for L in grid[::8]])
    assert np.allclose(curve[::8], dense, rtol=1e-6)
    assert idx == int(np.argmin(curve)) and lam == grid[idx]
    assert np.allclose(grid, ps.sigma[0] * 10.0 ** np.linspace(-16, 0, 321), rtol=1e-15)


def test_rho_eta_match_explicit_solution():
    _, _, g = _gkb(l=20, seed=4)
    C = g.C()
    ps = R.projected_svd(C, g.beta1)
    b = np.zeros(C.shape[0])
    b[0] = g.beta1
    for t in (-6, -3, -1):
        lam = ps.sigma[0] * 10.0 ** t
        y = pins.tikhonov_lstsq(C, b, lam)
        assert R.rho2_proj(ps, lam)[0] == pytest.approx(np.sum((C @ y - b) ** 2), rel=1e-8)
        assert R.eta2_proj(ps, lam)[0] == pytest.approx(np.sum(y ** 2), rel=1e-8)


def test_hkt_solution_equals_lstsq_and_normal_equations():
    _, _, g = _gkb(l=20, seed=5)
    C = g.C()
    ps = R.projected_svd(C, g.beta1)
    b = np.zeros(C.shape[0])
    b[0] = g.beta1
    for t in (-5, -3, -1):
        lam = ps.sigma[0] * 10.0 ** t
        y = R.hkt_solve_proj(ps, lam)
        y_ls = pins.tikhonov_lstsq(C, b, lam)
        y_ne = np.linalg.solve(C.T @ C + lam * lam * np.eye(ps.l), C.T @ b)  # Alg. 4 step 9
        assert np.linalg.norm(y - y_ls) / np.linalg.norm(y_ls) < 1e-12
        assert np.linalg.norm(y - y_ne) / np.linalg.norm(y_ne) < 1e-9


def test_full_rank_projection_equals_full_tikhonov_and_tsvd():
    # l = N: projected HKT / Ine-TSVD reduce to full Tikhonov / TSVD (Remark, Props.)
    rng = np.random.default_rng(6)
    n = 40
    A = mq.assemble(rng.uniform(0, 1, (n, 3)), 25, 0.05, 2.0)
    f = rng.normal(size=n)
    g = G.gkb(A, None, f, n)
    fs = R.full_svd(A, f)
    for t in (-4, -2, -1):
        lam = fs.sigma[0] * 10.0 ** t
        h = R.hkt(g, "fixed", lam)
        ref = np.linalg.solve(A.T @ A + lam * lam * np.eye(n), A.T @ f)  # normal equations
        full = R.tikhonov_full(A, f, "fixed", lam, fs=fs)["coef"]
        assert np.linalg.norm(h["coef"] - ref) / np.linalg.norm(ref) < 1e-9
        assert np.linalg.norm(full - ref) / np.linalg.norm(ref) < 1e-9
    for k in (3, 10, 25):
        it = R.ine_tsvd(g, rank=k)["coef"]
        ref = pins.tsvd_via_eigh(A, f, k)
        assert np.linalg.norm(it - ref) / np.linalg.norm(ref) < 1e-8
        assert np.linalg.norm(R.tsvd_full(A, f, rank=k, fs=fs)["coef"] - ref) / np.linalg.norm(ref) < 1e-8


def test_full_gcv_matches_dense_hat_matrix():
    rng = np.random.default_rng(7)
    n = 30
    A = mq.assemble(rng.uniform(0, 1, (n, 3)), 20, 0.1, 2.0)
    f = rng.normal(size=n)
    fs = R.full_svd(A, f)
    for t in (-6, -3, -1):
        lam = fs.sigma[0] * 10.0 ** t
        H = pins.hat_matrix(A, lam)
        r = f - H @ f
        ref = float(r @ r) / (n - np.trace(H)) ** 2
        assert R.gcv_full(fs, lam)[0] == pytest.approx(ref, rel=1e-8)


def test_rank_gcv_brute_force():
    _, _, g = _gkb(l=25, seed=8)
    ps = R.projected_svd(g.C(), g.beta1)
    k, curve = R.gcv_rank_proj(ps)
    b = np.zeros(ps.l + 1)
    b[0] = g.beta1
    C = g.C()
    for kk in (1, 5, 12, 25):
        y = R.tsvd_solve_proj(ps, kk)
        # residual of the rank-kk projected TSVD over the remaining degrees of freedom
        ref = np.sum((C @ y - b) ** 2) / (ps.l + 1 - kk) ** 2
        assert curve[kk - 1] == pytest.approx(ref, rel=1e-8)
    assert k == int(np.argmin(curve)) + 1


def test_curvature_of_circles():
    t = np.linspace(0, 2 * math.pi, 401)
    h = t[1] - t[0]
    for R0 in (0.5, 2.0):
        k_ccw = R.lcurve_curvature(R0 * np.cos(t), R0 * np.sin(t), h)
        k_cw = R.lcurve_curvature(R0 * np.cos(t), -R0 * np.sin(t), h)
        assert np.allclose(k_ccw, 1 / R0, rtol=1e-4) and np.allclose(k_cw, -1 / R0, rtol=1e-4)


def test_lcurve_corner_near_optimal_lambda():
    # synthetic discrete ill-posed problem satisfying the discrete Picard condition
    rng = np.random.default_rng(9)
    n = 60
    U, _ = np.linalg.qr(rng.normal(size=(n, n)))
    V, _ = np.linalg.qr(rng.normal(size=(n, n)))
    s = 10.0 ** (-np.arange(n) / 4.0)
    A = U @ np.diag(s) @ V.T
    x_true = V @ (s ** 0.5 * rng.choice([-1, 1], n))
    b = A @ x_true + 1e-6 * rng.normal(size=n)
    g = G.gkb(A, None, b, n)
    h = R.hkt(g, "lcurve")
    grid = h["grid"]
    errs = [np.linalg.norm(R.hkt(g, "fixed", L)["coef"] - x_true) for L in grid]
    best = int(np.argmin(errs))
    assert abs(h["index"] - best) <= 40  # within two decades on the 0.05-decade grid
    # far better than either end of the grid (no / full regularization)
    assert errs[h["index"]] < 0.25 * min(errs[0], errs[-1])


def test_lcurve_ignores_stationary_stretch():
    # l < N with noisy data: for lambda far below every s~_i, rho -> f~_{l+1} and
    # eta -> |y_0| are constant to rounding; those samples are not candidates
    rng = np.random.default_rng(12)
    n = 60
    U, _ = np.linalg.qr(rng.normal(size=(n, n)))
    V, _ = np.linalg.qr(rng.normal(size=(n, n)))
    A = U @ np.diag(10.0 ** (-np.arange(n) / 8.0)) @ V.T
    f = A @ rng.normal(size=n) + 1e-3 * rng.normal(size=n)
    g = G.gkb(A, None, f, 20)
    h = R.hkt(g, "lcurve")
    t = R.grid_t()
    s_min = h["ps"].sigma[-1] / h["ps"].sigma[0]
    below = t[1:-1] < np.log10(s_min) - 3.0
    assert np.all(np.isneginf(h["curve"][below]))
    assert t[h["index"]] > np.log10(s_min) - 3.0


def test_full_svd_numerical_rank_by_construction():
    assert pins.pin_full_rank(R.full_svd, np.random.default_rng(13))


def test_full_tsvd_gcv_rank_curve_brute_force():
    assert pins.pin_tsvd_gcv_curve(R.tsvd_full, np.random.default_rng(14))
