"""Oracle pins for the end-to-end methods on small MQ Helmholtz problems."""
import numpy as np

import workloads as w
from oracle import evaluate as E
from oracle import gkb as G
from oracle import mq
from oracle import regularize as R


def _cube(n_side=6, c=0.3, k=2.0):
    ns = w.cube_grid(n_side)
    A = mq.assemble(ns.X, ns.n_interior, c, k)
    f = w.plane_wave_rhs(ns, k)
    return ns, A, f


def test_reconstruction_at_boundary_nodes_equals_boundary_rows():
    ns, A, f = _cube()
    coef = np.random.default_rng(0).normal(size=ns.n)
    ub = E.reconstruct(coef, ns.X, ns.X[ns.n_interior:], 0.3)
    assert np.allclose(ub, (A @ coef)[ns.n_interior:], rtol=1e-13)
    # interior rows are L Phi, not Phi: the reconstruction uses the basis itself
    ui = E.reconstruct(coef, ns.X, ns.X[: ns.n_interior], 0.3)
    assert not np.allclose(ui, (A @ coef)[: ns.n_interior])


def test_eps_form_gives_same_u():
    # random (asymmetric) nodes: the symmetric grid makes GKB rounding-sensitive
    ns = w.cube_faces_random(216, 0.45, np.random.Generator(np.random.PCG64(1)))
    c = 0.3
    A = mq.assemble(ns.X, ns.n_interior, c, 2.0)
    f = w.plane_wave_rhs(ns, 2.0)
    Ae = mq.assemble(ns.X, ns.n_interior, c, 2.0, form="eps")
    P = w.test_points(ns, 200)
    g = G.gkb(A, None, f, 40)
    ge = G.gkb(Ae, None, f, 40)
    lam = 1e-4 * np.linalg.norm(A, 2)
    u_c = E.reconstruct(R.hkt(g, "fixed", lam)["coef"], ns.X, P, c)
    u_e = E.reconstruct(R.hkt(ge, "fixed", lam / c)["coef"], ns.X, P, c, form="eps")
    assert np.max(np.abs(u_c - u_e)) / np.max(np.abs(u_c)) < 1e-9


def test_plane_wave_error_decreases_with_steps():
    # accuracy of HKT (L-curve) against the exact plane wave improves with l until it plateaus
    ns, A, f = _cube(8)
    P = w.test_points(ns, 300)
    u = w.plane_wave(P, 2.0)
    g = G.gkb(A, None, f, ns.n)
    res = []
    for l in (10, 40, 160):
        gl = G.GKBResult(g.W, g.Z, g.alpha, g.beta, l, 0, g.c_hat)
        res.append(E.rel_error(u, E.reconstruct(R.hkt(gl, "lcurve")["coef"], ns.X, P, 0.3)))
    assert res[0] > 5 * res[1] and res[1] > res[2]
    assert res[2] < 2e-2


def test_full_tikhonov_recovers_plane_wave():
    ns, A, f = _cube(8)
    P = w.test_points(ns, 300)
    u = w.plane_wave(P, 2.0)
    t = R.tikhonov_full(A, f)
    assert E.rel_error(u, E.reconstruct(t["coef"], ns.X, P, 0.3)) < 2e-2


def test_rel_error_definition():
    u = np.array([1.0, -2.0, 0.5])
    ua = np.array([1.1, -2.0, 0.0])
    assert E.rel_error(u, ua) == 0.25
