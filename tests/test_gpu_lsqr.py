"""GPU: LSQR early stopping (Sec. 3.4) against the FP64 oracle.

The projected part is compared on identical inputs (the GPU's own alpha,
beta and Z fed to the oracle): rho_k and eta_k rel <= 1e-10, the same stopping
index, the same iterate.  End to end against the oracle's own GKB run the
tolerance follows the GKB parity rule (early steps, rel <= 1e-10 on a
well-separated problem).
"""
import numpy as np
import pytest

import workloads as w
from oracle import gkb as OG
from oracle import lsqr as OL
from oracle import mq as OM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09798_gb300 import rbfkr
    return rbfkr


@pytest.fixture(scope="module")
def ctx(R):
    c = R.Context(0)
    yield c
    c.close()


def _run(ctx, R, n, seed, c, k, L):
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = w.cube_faces_random(n, 0.3, rng)
    f = w.plane_wave_rhs(ns, k)
    nodes = torch.as_tensor(ns.soa(), device="cuda")
    lda = R.padded_lda(ns.n, R.RBF_FP64)
    A = torch.empty((ns.n, lda), dtype=torch.float64, device="cuda")
    op = ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, c, k, R.RBF_ASSEMBLED, R.RBF_FP64, A=A, lda=lda)
    ctx.rbf_assemble(op)
    st, W, Z, al, be = R.make_state(torch, ns.n, L)
    ctx.rbf_gkb(op, torch.as_tensor(f, device="cuda"), L, st)
    return ns, f, st, Z, al, be


@pytest.mark.parametrize("rule", ["lcurve", "gcv"])
def test_lsqr_projected_part_matches_oracle(ctx, R, rule):
    ns, f, st, Z, al, be = _run(ctx, R, 800, 41, 0.3, 2.0, 60)
    l = st.steps_done
    a, b = al.cpu().numpy(), be.cpu().numpy()
    rho, eta, ys = OL.lsqr_sequence(a, b, l)
    k_or, curve_or = OL.choose_k(rho, eta, l, rule)
    coef = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    curve = torch.empty(l, dtype=torch.float64, device="cuda")
    info = ctx.rbf_lsqr(st, R.RBF_LCURVE if rule == "lcurve" else R.RBF_GCV, 0, coef, curve)
    assert info.rank == k_or
    assert abs(info.rho - rho[k_or - 1]) <= 1e-10 * rho[k_or - 1]
    assert abs(info.eta - eta[k_or - 1]) <= 1e-10 * eta[k_or - 1]
    x_ref = Z[:k_or].cpu().numpy().T @ ys[k_or - 1]
    assert np.max(np.abs(coef.cpu().numpy() - x_ref)) <= 1e-10 * np.max(np.abs(x_ref))
    cg = curve.cpu().numpy()
    fin = np.isfinite(curve_or)
    assert np.array_equal(fin, np.isfinite(cg))
    assert np.max(np.abs(cg[fin] - curve_or[fin]) / (np.abs(curve_or[fin]) + 1e-300)) <= 1e-7


def test_lsqr_every_k_and_fixed(ctx, R):
    ns, f, st, Z, al, be = _run(ctx, R, 500, 42, 0.4, 3.0, 30)
    l = st.steps_done
    rho, eta, ys = OL.lsqr_sequence(al.cpu().numpy(), be.cpu().numpy(), l)
    coef = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    for k in (1, 2, 17, l):
        info = ctx.rbf_lsqr(st, R.RBF_FIXED, k, coef)
        assert info.rank == k
        assert abs(info.rho - rho[k - 1]) <= 1e-10 * rho[k - 1] + 1e-300
        assert abs(info.eta - eta[k - 1]) <= 1e-10 * eta[k - 1]
    with pytest.raises(R.RbfError):
        ctx.rbf_lsqr(st, R.RBF_FIXED, l + 1, coef)


def test_lsqr_end_to_end_against_oracle_gkb(ctx, R):
    ns, f, st, Z, al, be = _run(ctx, R, 700, 43, 0.3, 2.0, 12)
    A = OM.assemble(ns.X, ns.n_interior, 0.3, 2.0)
    g = OG.gkb(A, None, f, 12)
    out = OL.lsqr_solve(g, "fixed", k=12)
    coef = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    info = ctx.rbf_lsqr(st, R.RBF_FIXED, 12, coef)
    assert abs(info.rho - out["rho"][11]) <= 1e-10 * out["rho"][11]
    assert np.max(np.abs(coef.cpu().numpy() - out["coef"])) <= 1e-9 * np.max(np.abs(out["coef"]))
