"""The stop network as a C caller uses it: rbf_stopnet_load reads the shipped
binary file into a caller-owned device buffer (no Python loader involved), and
the learned-stop HKT driven by it must equal the run driven by the .npz loaded
in Python, bitwise; rbf_stopnet_save must write the same bytes back; a damaged
file is refused."""
import os

import numpy as np
import pytest

import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
PKG = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2511_09798_gb300")
BIN = os.path.join(PKG, "stopnet_weights.bin")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09798_gb300 import rbfkr
    return rbfkr


def test_c_loaded_network_drives_the_learned_stop(R, tmp_path):
    ctx = R.Context(0)
    storage = torch.empty(R.RBF_STOPNET_DEVICE_FLOATS, dtype=torch.float32, device="cuda")
    net_c = ctx.rbf_stopnet_load(BIN, storage)
    # a Gaussian problem of the training distribution, mixed precision, matrix-free
    rng = np.random.Generator(np.random.PCG64(71))
    ns = w.cube_faces_random(3000, 0.3, rng)
    c, k = 0.3, 4.0
    f = torch.as_tensor(w.gaussian_rhs(ns, 0.5, k, (0.5, 0.5, 0.5)), device="cuda")
    nodes = torch.as_tensor(ns.soa(), device="cuda")
    op = ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, c, k, R.RBF_MATRIX_FREE, R.RBF_MIXED)
    st1 = R.make_state(torch, ns.n, net_c.l_max)[0]
    coef1 = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    info1 = ctx.rbf_learned_hkt(op, f, net_c, st1, coef1)
    from paper_2511_09798_gb300 import learned
    net_py = learned.StopNet.load(torch, os.path.join(PKG, "stopnet_weights.npz"))
    st2 = R.make_state(torch, ns.n, net_c.l_max)[0]
    coef2 = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    info2 = learned.solve(ctx, op, f, net_py, st2, coef2)
    assert (info1.l_pred, info1.accepted, info1.steps) == (info2.l_pred, info2.accepted, info2.steps)
    assert info1.t_pred == info2.t_pred and info1.solve.lambda_ == info2.solve.lambda_
    assert torch.equal(coef1, coef2)
    # the C save writes the same bytes as the shipped file
    out = str(tmp_path / "net.bin")
    ctx.rbf_stopnet_save(net_c, out)
    assert open(out, "rb").read() == open(BIN, "rb").read()
    # damaged files are refused
    bad = str(tmp_path / "bad.bin")
    open(bad, "wb").write(open(BIN, "rb").read()[:-4])
    with pytest.raises(R.RbfError) as e:
        ctx.rbf_stopnet_load(bad, storage)
    assert e.value.status == R.RBF_ERR_INVALID
    open(bad, "wb").write(b"XBFSTOP1" + open(BIN, "rb").read()[8:])
    with pytest.raises(R.RbfError):
        ctx.rbf_stopnet_load(bad, storage)
    ctx.close()


def test_init_from_host_arrays_matches_load(R):
    ctx = R.Context(0)
    z = np.load(os.path.join(PKG, "stopnet_weights.npz"))
    s1 = torch.empty(R.RBF_STOPNET_DEVICE_FLOATS, dtype=torch.float32, device="cuda")
    s2 = torch.empty_like(s1)
    a = ctx.rbf_stopnet_load(BIN, s1)
    b = ctx.rbf_stopnet_init(s2, z["params"], z["feat_mean"], z["feat_std"],
                             np.concatenate([z["out_mean"], z["out_std"]]), z["rules"], z["tols"])
    assert torch.equal(s1, s2)
    for name in ("l_min", "l_max", "window", "fallback_rule", "accept_tol", "t_min", "t_max", "z_max", "feat_steps"):
        assert getattr(a, name) == getattr(b, name), name
    with pytest.raises(R.RbfError):  # l_max beyond 1023
        ctx.rbf_stopnet_init(s2, z["params"], None, None, [0, 0, 1, 1], [10, 2000, 5, 0], [1.0, -16, 0, 6])
    ctx.close()
