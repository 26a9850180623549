"""Oracle pins: Golub-Kahan bidiagonalization (Algorithm 1)."""
import numpy as np
import pytest

import pins
import workloads as w
from oracle import gkb as G
from oracle import mq


def _mq_problem(n=200, ni=140, c=0.2, k=3.0, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (n, 3))
    A = mq.assemble(X, ni, c, k)
    f = rng.normal(size=n)
    return A, f


@pytest.mark.parametrize("reorth", ["mgs2", "cgs2"])
def test_gkb_relations_mq(reorth):
    A, f = _mq_problem()
    g = G.gkb(A, None, f, 60, reorth=reorth)
    assert g.steps_done == 60
    pins.pin_gkb_relations(A, f, g)


def test_gkb_relations_cube_workload():
    ns = w.cube_grid(10)
    A = mq.assemble(ns.X, ns.n_interior, 0.3, 2.0)
    f = w.plane_wave_rhs(ns, 2.0)
    g = G.gkb(A, None, f, 40)
    pins.pin_gkb_relations(A, f, g)


def test_matrix_free_callables_equal_dense():
    A, f = _mq_problem(80, 50)
    g1 = G.gkb(A, None, f, 20)
    g2 = G.gkb(lambda x: A @ x, lambda y: A.T @ y, f, 20)
    assert np.array_equal(g1.alpha, g2.alpha) and np.array_equal(g1.beta, g2.beta)


def test_full_run_ritz_values_equal_svd():
    # l = N: the Ritz values are the singular values of A (Remark on projected formulations)
    rng = np.random.default_rng(1)
    for A in (rng.normal(size=(40, 40)), mq.assemble(rng.uniform(0, 1, (40, 3)), 25, 0.05, 2.0)):
        f = rng.normal(size=40)
        g = G.gkb(A, None, f, 40)
        s_ritz = pins.tgk_singular_values(g.C())
        s_full = np.linalg.svd(A, compute_uv=False)
        assert np.max(np.abs(s_ritz - s_full)) / s_full[0] < 1e-12


def test_top_ritz_values_converge():
    A, f = _mq_problem(300, 200, c=0.3)
    s_full = np.linalg.svd(A, compute_uv=False)
    errs = []
    for l in (10, 20, 40):
        g = G.gkb(A, None, f, l)
        s = pins.tgk_singular_values(g.C())
        errs.append(np.max(np.abs(s[:8] - s_full[:8]) / s_full[:8]))
    assert errs[0] > 1e-3 and errs[0] > errs[1] > errs[2] and errs[2] < 1e-12


def test_rank_deficient_breaks_down_beta():
    rng = np.random.default_rng(2)
    n, r = 60, 12
    U, _ = np.linalg.qr(rng.normal(size=(n, r)))
    V, _ = np.linalg.qr(rng.normal(size=(n, r)))
    A = U @ np.diag(np.logspace(0, -3, r)) @ V.T
    f = A @ rng.normal(size=n)
    g = G.gkb(A, None, f, 30)
    assert g.steps_done == r and g.breakdown == 2
    assert g.beta[r] == 0.0 and np.all(g.W[:, r] == 0.0)
    pins.pin_gkb_relations(A, f, g, tol=1e-11)


def test_alpha_breakdown_when_f_in_left_null_space():
    # At step 1 no scale estimate of |A| exists yet (c_hat = 0), so only an exact
    # zero alpha_1 stops the run: A^T f = 0 exactly here.
    rng = np.random.default_rng(3)
    n = 30
    A = rng.normal(size=(n, n))
    A[20:] = 0.0
    f = np.zeros(n)
    f[25] = 1.0
    g = G.gkb(A, None, f, 10)
    assert g.steps_done == 0 and g.breakdown == 1


def test_alpha_breakdown_later_step():
    # A^T w_2 has no component outside span{z_1}: alpha_2 falls below tau
    n = 10
    A = np.zeros((n, n))
    A[0, 0], A[1, 0] = 3.0, 4.0
    f = np.zeros(n)
    f[0] = 1.0
    g = G.gkb(A, None, f, 5)
    assert g.steps_done == 1 and g.breakdown == 1
    assert g.alpha[0] == pytest.approx(3.0) and g.beta[1] == pytest.approx(4.0)


def test_zero_rhs():
    A, _ = _mq_problem(20, 10)
    g = G.gkb(A, None, np.zeros(20), 5)
    assert g.steps_done == 0


def test_breakdown_threshold_rule():
    # tau = 64 N eps c_hat: a beta just below tau stops the run, just above does not
    n = 8
    eps = np.finfo(float).eps
    # span{e_0, e_1} is invariant: with beta_2 above tau the run continues to
    # step 2 and stops there on beta_3 = 0; below tau it stops at step 1.
    for factor, expect_done in ((0.5, 1), (2.0, 2)):
        A = np.eye(n)
        A[1, 0] = factor * 64 * n * eps  # beta_2 = this value, c_hat ~ 1
        f = np.zeros(n)
        f[0] = 1.0
        g = G.gkb(A, None, f, 3)
        assert g.steps_done == expect_done and g.breakdown == 2
