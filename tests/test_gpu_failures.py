"""GPU: failure paths, exercised without faulting, trapping or hanging the GPU.

* A device-side wait (the grid barrier of the half-step kernel) allowed one
  poll gives up: the run stops, the call returns RBF_ERR_TIMEOUT, the same
  context still runs calls without device-side waits, and a new context
  solves the same problem correctly.
* A workspace cap below what a call needs gives RBF_ERR_OOM.
* NaN or Inf in f, or NaN in the matrix, stop GKB with breakdown 3 and the
  steps completed before it.
"""
import numpy as np
import pytest

import workloads as w
from oracle import gkb as OG
from oracle import mq as OM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C_, K_ = 0.3, 2.0


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09798_gb300 import rbfkr
    return rbfkr


def _nodes(n=600, ni=400, seed=7):
    rng = np.random.default_rng(seed)
    return w.NodeSet(rng.uniform(0, 1, (n, 3)), ni, "cube", f"rand{n}")


def _assembled(ctx, R, ns):
    lda = R.padded_lda(ns.n, R.RBF_FP64)
    A = torch.empty((ns.n, lda), dtype=torch.float64, device="cuda")
    nodes = torch.as_tensor(ns.soa(), device="cuda")
    op = ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, C_, K_, R.RBF_ASSEMBLED, R.RBF_FP64, R.RBF_FORM_C,
                               A, lda)
    ctx.rbf_assemble(op)
    return op, A, nodes


def test_wait_budget_timeout_leaves_device_usable(R):
    ns = _nodes()
    f_np = w.plane_wave_rhs(ns, K_)
    f = torch.as_tensor(f_np, device="cuda")
    Ah = OM.assemble(ns.X, ns.n_interior, C_, K_)
    tiny = R.Context(0, wait_budget=1)
    try:
        op, A, nodes = _assembled(tiny, R, ns)
        st, *_ = R.make_state(torch, ns.n, 40)
        with pytest.raises(R.RbfError) as e:
            tiny.rbf_gkb(op, f, 40, st)
        assert e.value.status == R.RBF_ERR_TIMEOUT
        # no device-side wait in a product: the context still works
        x = torch.ones(ns.n, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        tiny.rbf_matvec(op, 0, x, y)
        torch.cuda.synchronize()
        ref = Ah @ np.ones(ns.n)
        assert np.max(np.abs(y.cpu().numpy() - ref)) / np.max(np.abs(ref)) < 1e-14
    finally:
        tiny.close()
    normal = R.Context(0)
    try:
        op, A, nodes = _assembled(normal, R, ns)
        st, W, Z, al, be = R.make_state(torch, ns.n, 20)
        normal.rbf_gkb(op, f, 20, st)
        g = OG.gkb(Ah, None, f_np, 20)
        assert st.steps_done == g.steps_done and st.breakdown == 0
        assert abs(al.cpu().numpy()[0] - g.alpha[0]) / g.alpha[0] < 1e-12
        assert abs(be.cpu().numpy()[1] - g.beta[1]) / g.beta[1] < 1e-12
    finally:
        normal.close()


def test_workspace_cap_gives_oom(R):
    ns = _nodes()
    ctx = R.Context(0, workspace_cap=4096)
    try:
        op, A, nodes = _assembled(ctx, R, ns)
        st, *_ = R.make_state(torch, ns.n, 10)
        with pytest.raises(R.RbfError) as e:
            ctx.rbf_gkb(op, torch.as_tensor(w.plane_wave_rhs(ns, K_), device="cuda"), 10, st)
        assert e.value.status == R.RBF_ERR_OOM
        assert "cap" in str(e.value)
    finally:
        ctx.close()


def test_nonfinite_inputs_stop_cleanly(R):
    ns = _nodes()
    ctx = R.Context(0)
    try:
        op, A, nodes = _assembled(ctx, R, ns)
        f_np = w.plane_wave_rhs(ns, K_)
        for bad in (np.nan, np.inf):
            fb = f_np.copy()
            fb[17] = bad
            st, *_ = R.make_state(torch, ns.n, 10)
            ctx.rbf_gkb(op, torch.as_tensor(fb, device="cuda"), 10, st)
            assert st.steps_done == 0 and st.breakdown == 3, (bad, st.steps_done, st.breakdown)
        # NaN in the matrix: beta_1 = |f| is finite, alpha_1 = |A^T w_1| is not
        A[5, 3] = float("nan")
        st, *_ = R.make_state(torch, ns.n, 10)
        ctx.rbf_gkb(op, torch.as_tensor(f_np, device="cuda"), 10, st)
        assert st.steps_done == 0 and st.breakdown == 3
        # the context keeps working once the matrix is clean again
        ctx.rbf_assemble(op)
        st, *_ = R.make_state(torch, ns.n, 10)
        ctx.rbf_gkb(op, torch.as_tensor(f_np, device="cuda"), 10, st)
        assert st.steps_done == 10 and st.breakdown == 0
    finally:
        ctx.close()


def test_batched_nonfinite_instance_stops_alone(R):
    rng = np.random.default_rng(11)
    sets = [w.cube_faces_random(500, 0.3, rng), w.cube_faces_random(700, 0.3, rng),
            w.sphere_fibonacci_ball(100, 300, seed=5)]
    cs, ks = [0.3, 0.25, 0.2], [2.0, 3.0, 4.0]
    fs = [w.plane_wave_rhs(s, k) for s, k in zip(sets, ks)]
    fs[1] = fs[1].copy()
    fs[1][42] = np.nan
    L = 12
    ctx = R.Context(0)
    try:
        bt, keep = R.make_batch(torch, sets, cs, ks, fs, L, "cuda")
        ctx.rbf_batch_gkb(bt, L)
        assert bt.breakdown[1] == 3 and bt.steps_done[1] == 0
        for b in (0, 2):
            assert bt.breakdown[b] == 0 and bt.steps_done[b] == L
    finally:
        ctx.close()
