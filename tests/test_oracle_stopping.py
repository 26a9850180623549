"""Oracle pins for the learned stop's features and error table.

Pins are independent of the oracle's formulas: the residual features are
checked against least squares on the full matrix over the Krylov subspace
(the GKB relation A Z_i = W_{i+1} C_i, Algorithm 1), the singular-value
features against the Golub-Kahan tridiagonal eigenvalues, the error table
against a direct solve when the Krylov space is the whole space.
"""
import numpy as np

import workloads as w
from oracle import gkb as OG
from oracle import mq as OM
from oracle import stopping as OS
from tests import pins


def _small_problem(n=90, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = w.cube_faces_random(n, 0.35, rng)
    A = OM.assemble(ns.X, ns.n_interior, 0.4, 2.0)
    f = w.plane_wave_rhs(ns, 2.0)
    return ns, A, f


def test_residual_features_equal_full_least_squares():
    ns, A, f = _small_problem()
    g = OG.gkb(A, None, f, 12)
    feat = OS.stop_features(g.alpha, g.beta, 10)
    for i in range(1, 11):
        Zi = g.Z[:, :i]
        x = np.linalg.lstsq(A @ Zi, f, rcond=None)[0]
        rho = np.linalg.norm(A @ Zi @ x - f)
        assert abs(10.0 ** feat[9 + i] - rho / np.linalg.norm(f)) <= 1e-8 * rho / np.linalg.norm(f), i
    # residuals cannot grow with i (nested subspaces)
    assert np.all(np.diff(feat[10:]) <= 1e-12)


def test_singular_value_features_match_tridiagonal_eigenvalues():
    ns, A, f = _small_problem(seed=4)
    g = OG.gkb(A, None, f, 10)
    feat = OS.stop_features(g.alpha, g.beta, 10)
    s = pins.tgk_singular_values(g.C())
    assert abs(feat[0] - np.log10(s[0])) < 1e-12
    assert np.max(np.abs(feat[1:10] - np.log10(s[1:10] / s[0]))) < 1e-9


def test_short_runs_and_zero_residual():
    # A diagonal: f in the span of two eigenvectors -> GKB ends after 2 steps
    # with beta_3 = 0 and a zero least-squares residual from step 2 on.
    n = 20
    A = np.diag(np.arange(1.0, n + 1))
    f = np.zeros(n)
    f[0], f[1] = 1.0, 2.0
    g = OG.gkb(A, None, f, 10)
    assert g.steps_done == 2
    feat = OS.stop_features(g.alpha, g.beta, 2)
    assert np.all(feat[2:10] == OS.NEG)
    assert feat[11] == OS.NEG and np.all(feat[12:] == OS.NEG)
    # the first residual is |f - proj| with one Krylov vector: by hand
    z1 = A.T @ f / np.linalg.norm(A.T @ f)
    p = A @ z1
    r = f - p * (p @ f) / (p @ p)
    assert abs(10.0 ** feat[10] - np.linalg.norm(r) / np.linalg.norm(f)) < 1e-12


def test_error_table_full_space_equals_direct_solve():
    rng = np.random.Generator(np.random.PCG64(8))
    X = rng.uniform(0, 1, (14, 3))
    n_int = 6
    A = OM.assemble(X, n_int, 0.6, 1.5)
    f = rng.normal(size=14)
    g = OG.gkb(A, None, f, 14)
    assert g.steps_done == 14
    P = rng.uniform(0, 1, (40, 3))
    uref = rng.normal(size=40)
    E = OS.error_table(g, X, 0.6, P, uref, [14], [-30.0])
    coef = np.linalg.solve(A, f)
    D = np.sqrt(((P[:, None, :] - X[None, :, :]) ** 2).sum(-1) + 0.36)
    e_direct = np.max(np.abs(D @ coef - uref)) / np.max(np.abs(uref))
    assert abs(E[0, 0] - e_direct) <= 1e-6 * e_direct
