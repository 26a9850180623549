"""GPU: the one-call solve helper (assemble -> GKB -> HKT -> evaluate) on a
context whose lambda grid is larger than the default 321 points.  The GCV curve
buffer must hold the context's J values (a buffer sized for 321 would be
overrun), and the choice must match the oracle's GCV on the same grid."""
import numpy as np
import pytest

import workloads as w
from oracle import evaluate as OE
from oracle import gkb as OG
from oracle import mq as OM
from oracle import regularize as OR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09798_gb300 import rbfkr
    return rbfkr


def test_pipeline_solve_on_a_641_point_grid(R):
    from paper_2511_09798_gb300 import pipeline as P
    ns = w.cube_faces_random(600, 0.35, np.random.Generator(np.random.PCG64(41)))
    c, k, steps, J = 0.3, 2.0, 30, 641
    f = w.plane_wave_rhs(ns, k)
    pts = w.test_points(ns, 300)
    ctx = R.Context(0, grid_j=J)
    assert ctx.grid_j == J
    prob = P.to_device(torch, ns.soa(), f, pts, ns.n_interior, c, k)
    buf = P.allocate(torch, ctx, prob, steps, R.RBF_FP64, R.RBF_ASSEMBLED)
    assert buf.curve.numel() >= J
    # a guard value past the J curve entries must survive the solve
    guard = torch.full((buf.curve.numel() + 8,), 7.0, dtype=torch.float64, device="cuda")
    buf.curve = guard[:J]
    op, info = P.solve(ctx, prob, buf, steps, rule=R.RBF_GCV)
    torch.cuda.synchronize()
    assert torch.all(guard[J:] == 7.0)
    g = OG.gkb(OM.assemble(ns.X, ns.n_interior, c, k), None, f, steps)
    assert buf.state.steps_done == g.steps_done
    h = OR.hkt(g, "gcv", J=J)
    assert np.allclose(buf.curve.cpu().numpy(), h["curve"], rtol=1e-9, atol=0)
    if info.index != h["index"]:
        gv = OR.gcv_proj(h["ps"], np.array([info.lambda_, h["lam"]]))
        assert gv[0] <= (1 + 1e-10) * gv[1]
    else:
        assert info.lambda_ == pytest.approx(h["lam"], rel=1e-13)
    # u at the oracle's lambda
    ctx.rbf_hkt(buf.state, R.RBF_FIXED, h["lam"], buf.coef)
    ctx.rbf_evaluate(op, buf.coef, prob.points, prob.m, buf.u)
    u_or = OE.reconstruct(h["coef"], ns.X, pts, c)
    assert np.max(np.abs(buf.u.cpu().numpy() - u_or)) / np.max(np.abs(u_or)) < 1e-10
    # the binding refuses a curve buffer shorter than the grid
    with pytest.raises(ValueError):
        ctx.rbf_hkt(buf.state, R.RBF_GCV, 0.0, buf.coef, torch.empty(321, dtype=torch.float64, device="cuda"))
    ctx.close()


def test_grid_of_one_or_two_points_is_rejected(R):
    for J in (1, 2):
        with pytest.raises(R.RbfError):
            R.Context(0, grid_j=J)
