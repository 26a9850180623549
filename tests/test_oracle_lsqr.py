"""Oracle pins for LSQR early stopping (Sec. 3.4).

The LSQR iterate is pinned against least squares on the full matrix over the
Krylov subspace, and against the direct solve when the subspace is the whole
space; the stopping rules against sequences whose answer is known by
construction.
"""
import numpy as np

import workloads as w
from oracle import gkb as OG
from oracle import lsqr as OL
from oracle import mq as OM


def test_iterates_minimise_the_residual_over_the_krylov_subspace():
    rng = np.random.Generator(np.random.PCG64(31))
    ns = w.cube_faces_random(120, 0.35, rng)
    A = OM.assemble(ns.X, ns.n_interior, 0.4, 3.0)
    f = w.plane_wave_rhs(ns, 3.0)
    g = OG.gkb(A, None, f, 25)
    rho, eta, ys = OL.lsqr_sequence(g.alpha, g.beta, 25)
    for k in (1, 4, 11, 25):
        Zk = g.Z[:, :k]
        c = np.linalg.lstsq(A @ Zk, f, rcond=None)[0]
        x_ref = Zk @ c
        x = Zk @ ys[k - 1]
        r_ref = np.linalg.norm(A @ x_ref - f)
        assert abs(rho[k - 1] - r_ref) <= 1e-8 * np.linalg.norm(f), k
        assert np.linalg.norm(x - x_ref) <= 1e-6 * np.linalg.norm(x_ref), k
        assert abs(eta[k - 1] - np.linalg.norm(x_ref)) <= 1e-6 * np.linalg.norm(x_ref), k
    assert np.all(np.diff(rho) <= 1e-12 * rho[0])  # nested subspaces


def test_full_space_iterate_is_the_solution():
    rng = np.random.Generator(np.random.PCG64(32))
    A = rng.normal(size=(12, 12)) + 6 * np.eye(12)
    f = rng.normal(size=12)
    g = OG.gkb(A, None, f, 12)
    out = OL.lsqr_solve(g, "fixed", k=12)
    assert np.max(np.abs(out["coef"] - np.linalg.solve(A, f))) < 1e-10 * np.max(np.abs(np.linalg.solve(A, f)))


def test_gcv_stops_where_the_residual_stops_falling():
    # rho drops by 10x per step up to k = 6, then stays: GCV = rho^2/((l+1)-k)^2
    # keeps falling while rho falls faster than the denominator and rises after
    l = 20
    rho = np.array([10.0 ** -(min(k, 6)) for k in range(1, l + 1)])
    eta = np.linspace(1, 2, l)
    k, g = OL.choose_k(rho, eta, l, "gcv")
    assert k == 6


def test_lcurve_finds_the_corner_of_an_l_shaped_sequence():
    # ln rho falls steeply while ln eta is flat (k <= 8), then ln rho is flat
    # while ln eta climbs: the corner is at k = 8
    l = 16
    k = np.arange(1, l + 1)
    lr = np.where(k <= 8, -1.0 * k, -8.0 - 0.01 * (k - 8))
    le = np.where(k <= 8, 0.01 * k, 0.08 + 1.0 * (k - 8))
    kk, curve = OL.choose_k(np.exp(lr), np.exp(le), l, "lcurve")
    assert kk == 8
    assert curve[7] > 0
