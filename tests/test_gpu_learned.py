"""GPU: the stop network's kernels against the FP64 oracle, the stop features,
the labelling error table, and the learned-stop HKT decision logic.

Tolerances: the network runs in FP32 (gradients accumulated in FP64), so
outputs and gradients agree with the FP64 oracle to rel <= 1e-4; features are
FP64 logs rounded to FP32 (abs <= 1e-5); the error table is FP64 throughout.
"""
import math

import numpy as np
import pytest

import workloads as w
from oracle import gkb as OG
from oracle import mlp as OMLP
from oracle import mq as OM
from oracle import regularize as OR
from oracle import stopping as OS

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


def _net_inputs(B, seed):
    rng = np.random.default_rng(seed)
    theta = OMLP.init_params(seed).astype(np.float32)
    theta += rng.normal(scale=0.05, size=theta.size).astype(np.float32)  # nonzero biases
    X = rng.normal(size=(B, 20)).astype(np.float32)
    T = rng.normal(size=(B, 2)).astype(np.float32)
    return theta, X, T


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("B", [1, 16, 300])
def test_forward_matches_oracle(ctx, B):
    theta, X, _ = _net_inputs(B, 1)
    y = torch.empty((B, 2), dtype=torch.float32, device="cuda")
    ctx.rbf_mlp_forward(_dev(theta), _dev(X), B, y)
    ref = OMLP.forward(theta.astype(np.float64), X.astype(np.float64))
    ref = ref[0] if isinstance(ref, tuple) else ref
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-4 * np.max(np.abs(ref))


@pytest.mark.parametrize("B", [5, 257])
def test_gradient_matches_oracle(ctx, B):
    theta, X, T = _net_inputs(B, 2)
    g = torch.empty(theta.size, dtype=torch.float32, device="cuda")
    loss = ctx.rbf_mlp_grad(_dev(theta), _dev(X), _dev(T), B, g)
    L, g_ref = OMLP.loss_and_grad(theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - L) <= 1e-4 * abs(L)
    gg = g.cpu().numpy()
    assert np.max(np.abs(gg - g_ref)) <= 1e-4 * np.max(np.abs(g_ref))
    # every layer's block, not just the largest entries
    for a, b in ((0, 2560), (2560, 2688), (2688, 19072), (19072, 19200), (19200, 19456), (19456, 19458)):
        assert np.linalg.norm(gg[a:b] - g_ref[a:b]) <= 1e-4 * np.linalg.norm(g_ref[a:b]) + 1e-12, (a, b)


def test_gradient_is_deterministic(ctx):
    theta, X, T = _net_inputs(100, 3)
    g1 = torch.empty(theta.size, dtype=torch.float32, device="cuda")
    g2 = torch.empty_like(g1)
    ctx.rbf_mlp_grad(_dev(theta), _dev(X), _dev(T), 100, g1, want_loss=False)
    ctx.rbf_mlp_grad(_dev(theta), _dev(X), _dev(T), 100, g2, want_loss=False)
    assert torch.equal(g1, g2)


def test_adam_matches_oracle(ctx):
    theta, X, T = _net_inputs(64, 4)
    rng = np.random.default_rng(5)
    m = rng.normal(scale=1e-3, size=theta.size).astype(np.float32)
    v = np.abs(rng.normal(scale=1e-5, size=theta.size)).astype(np.float32)
    g = rng.normal(scale=1e-2, size=theta.size).astype(np.float32)
    dp, dm, dv = _dev(theta.copy()), _dev(m.copy()), _dev(v.copy())
    ctx.rbf_mlp_adam(dp, dm, dv, _dev(g), 7, 1e-3)
    p_ref, m_ref, v_ref = OMLP.adam_step(theta.astype(np.float64), m.astype(np.float64), v.astype(np.float64),
                                         g.astype(np.float64), 7, lr=1e-3)
    step = np.abs(p_ref - theta)
    assert np.max(np.abs(dp.cpu().numpy() - p_ref) - 1e-3 * step) <= 1e-6 * np.max(np.abs(theta))
    # FP32 moments: b1 m + (1 - b1) g cancels for some entries, so the bound
    # is relative to the terms' size, not to the result
    assert np.max(np.abs(dm.cpu().numpy() - m_ref)) <= 1e-6 * (np.max(np.abs(m)) + np.max(np.abs(g)))
    assert np.max(np.abs(dv.cpu().numpy() - v_ref)) <= 1e-6 * (np.max(v) + np.max(g.astype(np.float64) ** 2))


def test_training_on_gpu_fits_a_teacher(ctx):
    """Adam on GPU drives the loss of a teacher network's targets down."""
    rng = np.random.default_rng(6)
    teacher = OMLP.init_params(11)
    X = rng.normal(size=(512, 20))
    Y = OMLP.forward(teacher, X)
    Y = (Y[0] if isinstance(Y, tuple) else Y).astype(np.float32)
    from paper_2511_09798_gb300 import learned
    p = _dev(learned.init_params(0))
    m, v, g = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
    dX, dY = _dev(X.astype(np.float32)), _dev(Y)
    l0 = ctx.rbf_mlp_grad(p, dX, dY, 512, g)
    for t in range(1, 401):
        ctx.rbf_mlp_train_step(p, m, v, t, 2e-3, dX, dY, 512, g)
    l1 = ctx.rbf_mlp_grad(p, dX, dY, 512, g)
    assert l1 < 0.05 * l0, (l0, l1)
    # the trained parameters reproduce the oracle's forward of themselves
    y = torch.empty((512, 2), dtype=torch.float32, device="cuda")
    ctx.rbf_mlp_forward(p, dX, 512, y)
    ref = OMLP.forward(p.cpu().numpy().astype(np.float64), X)
    ref = ref[0] if isinstance(ref, tuple) else ref
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-4 * np.max(np.abs(ref))


def _fp64_problem(n=700, seed=12, c=0.3, k=2.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = w.cube_faces_random(n, 0.3, rng)
    f = w.plane_wave_rhs(ns, k)
    return ns, f, c, k


def _gpu_gkb(ctx, R, ns, f, c, k, steps):
    nodes = _dev(ns.soa())
    lda = R.padded_lda(ns.n, R.RBF_FP64)
    A = torch.empty((ns.n, lda), dtype=torch.float64, device="cuda")
    op = ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, c, k, R.RBF_ASSEMBLED, R.RBF_FP64, A=A, lda=lda)
    ctx.rbf_assemble(op)
    st, *_ = R.make_state(torch, ns.n, steps)
    ctx.rbf_gkb(op, _dev(f), steps, st)
    return op, st


def test_stop_features_match_oracle(ctx, R):
    ns, f, c, k = _fp64_problem()
    op, st = _gpu_gkb(ctx, R, ns, f, c, k, 12)
    A = OM.assemble(ns.X, ns.n_interior, c, k)
    g = OG.gkb(A, None, f, 12)
    for j in (10, 4):
        feat = torch.empty(20, dtype=torch.float32, device="cuda")
        ctx.rbf_stop_features(st, j, feat)
        ref = OS.stop_features(g.alpha, g.beta, j)
        assert np.max(np.abs(feat.cpu().numpy() - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref))), j
    # standardisation on device
    mean = np.linspace(-1, 1, 20).astype(np.float32)
    std = np.linspace(0.5, 2, 20).astype(np.float32)
    feat = torch.empty(20, dtype=torch.float32, device="cuda")
    ctx.rbf_stop_features(st, 10, feat, _dev(mean), _dev(std))
    ref = (OS.stop_features(g.alpha, g.beta, 10) - mean) / std
    assert np.max(np.abs(feat.cpu().numpy() - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_evaluate_many_and_error_table_match_oracle(ctx, R):
    ns, f, c, k = _fp64_problem(n=500, seed=13)
    L = 30
    op, st = _gpu_gkb(ctx, R, ns, f, c, k, L)
    A = OM.assemble(ns.X, ns.n_interior, c, k)
    g = OG.gkb(A, None, f, L)
    P = w.test_points(ns, 333)
    uref = w.plane_wave(P, k)
    m = P.shape[0]
    G = torch.empty((L, m), dtype=torch.float64, device="cuda")
    ctx.rbf_evaluate_many(op, st.d_Z, ns.n, L, _dev(P.T), m, G)
    # column i against the single-vector reconstruction
    u1 = torch.empty(m, dtype=torch.float64, device="cuda")
    Zg = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    for i in (0, 17, L - 1):
        Zg.copy_(st._keep[1][i])
        ctx.rbf_evaluate(op, Zg, _dev(P.T), m, u1)
        assert torch.max(torch.abs(G[i] - u1)).item() <= 1e-12 * torch.max(torch.abs(u1)).item()
    ells = [5, 12, 30]
    stride = 16
    Jp = (321 - 1) // stride + 1
    err = torch.empty((len(ells), Jp), dtype=torch.float64, device="cuda")
    ctx.rbf_hkt_error_table(st, G, m, m, _dev(uref), ells, stride, err)
    tgrid = np.array([-16.0 + 16.0 * q * stride / 320 for q in range(Jp)])
    ref = OS.error_table(g, ns.X, c, P, uref, ells, tgrid)
    E = err.cpu().numpy()
    # the early steps of GKB agree to ~1e-12 between CGS2 and MGS2; lambda
    # below ~1e-10 s1 amplifies that by the conditioning of C_l
    tol = np.where(tgrid[None, :] >= -8.0, 1e-8, 1e-3)
    assert np.all(np.abs(E - ref) <= tol * np.maximum(ref, 1e-3)), np.max(np.abs(E - ref) / ref)


@pytest.mark.parametrize("ncoef", [1, 2, 3, 5, 11])
def test_evaluate_many_vector_counts(ctx, R, ncoef):
    """1, 2, 4 or 8 vectors per CTA (3, 5 and 11 leave a group part empty):
    every row equals the oracle's reconstruction and the single-vector call."""
    ns, f, c, k = _fp64_problem(n=389, seed=17)
    nodes = _dev(ns.soa())
    op = ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, c, k, R.RBF_MATRIX_FREE, R.RBF_FP64, R.RBF_FORM_EPS)
    rng = np.random.default_rng(ncoef)
    ldc = ns.n + 3
    Cf = rng.normal(size=(ncoef, ldc))
    P = w.test_points(ns, 211)
    m = P.shape[0]
    U = torch.empty((ncoef, m), dtype=torch.float64, device="cuda")
    ctx.rbf_evaluate_many(op, _dev(Cf), ldc, ncoef, _dev(P.T), m, U)
    Phi = OM.phi(OM.distances(P, ns.X), c) / c  # eps form scales by 1/c
    ref = Cf[:, :ns.n] @ Phi.T
    Ug = U.cpu().numpy()
    scale = np.abs(Cf[:, :ns.n]) @ np.abs(Phi.T)
    assert np.all(np.abs(Ug - ref) <= 1e-13 * scale), np.max(np.abs(Ug - ref) / scale)
    u1 = torch.empty(m, dtype=torch.float64, device="cuda")
    for i in sorted({0, ncoef - 1}):
        ctx.rbf_evaluate(op, _dev(np.ascontiguousarray(Cf[i, :ns.n])), _dev(P.T), m, u1)
        assert np.all(np.abs(Ug[i] - u1.cpu().numpy()) <= 1e-13 * scale[i])


def _constant_net(R, l_target, t_target, **kw):
    """A network whose output is exactly its last bias: W3 = 0 (the rest
    random), so the prediction is known: l = l_target, t = t_target."""
    from paper_2511_09798_gb300 import learned
    p = learned.init_params(9)
    p[19200:19456] = 0.0
    p[19456:19458] = 0.0
    kw.setdefault("z_max", 0.0)
    net = learned.StopNet(torch, p, np.zeros(20), np.ones(20), [math.log(l_target), t_target], [1.0, 1.0], **kw)
    return net


def test_learned_hkt_accepts_and_matches_fixed_solve(ctx, R):
    from paper_2511_09798_gb300 import learned
    ns, f, c, k = _fp64_problem(n=600, seed=14)
    net = _constant_net(R, 25, -6.0, l_min=10, l_max=40, window=5, accept_tol=1e30)
    nodes = _dev(ns.soa())
    lda = R.padded_lda(ns.n, R.RBF_FP64)
    A = torch.empty((ns.n, lda), dtype=torch.float64, device="cuda")
    op = ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, c, k, R.RBF_ASSEMBLED, R.RBF_FP64, A=A, lda=lda)
    ctx.rbf_assemble(op)
    st, *_ = R.make_state(torch, ns.n, 40)
    coef = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    info = learned.solve(ctx, op, _dev(f), net, st, coef)
    assert info.l_pred == 25 and abs(info.t_pred + 6.0) < 1e-6
    assert info.accepted == 1 and info.steps == 25 and st.steps_done == 25
    # the same solve from an uninterrupted 25-step run (resume equals it to rounding)
    st2, *_ = R.make_state(torch, ns.n, 40)
    ctx.rbf_gkb(op, _dev(f), 25, st2)
    coef2 = torch.empty_like(coef)
    i2 = ctx.rbf_hkt(st2, R.RBF_FIXED_T, -6.0, coef2)
    assert abs(i2.lambda_ - info.solve.lambda_) <= 1e-12 * i2.lambda_
    assert torch.max(torch.abs(coef - coef2)).item() <= 1e-8 * torch.max(torch.abs(coef2)).item()
    # and the FP64 oracle at the same (l, lambda)
    Ad = OM.assemble(ns.X, ns.n_interior, c, k)
    g = OG.gkb(Ad, None, f, 25)
    h = OR.hkt(g, "fixed", lam=info.solve.lambda_)
    assert np.max(np.abs(coef.cpu().numpy() - h["coef"])) <= 1e-6 * np.max(np.abs(h["coef"]))
    assert abs(info.solve.eta - np.linalg.norm(h["y"])) <= 1e-8 * np.linalg.norm(h["y"])
    # eta_change is the relative change against the 20-step solve at the same t
    g20 = OG.gkb(Ad, None, f, 20)
    ps20 = OR.projected_svd(g20.C(), g20.beta1)
    eta20 = np.linalg.norm(OR.hkt_solve_proj(ps20, ps20.sigma[0] * 1e-6))
    ref_change = abs(info.solve.eta - eta20) / info.solve.eta
    assert abs(info.eta_change - ref_change) <= 1e-6 * max(ref_change, 1e-12) + 1e-12


def test_learned_hkt_without_eta_test(ctx, R):
    from paper_2511_09798_gb300 import learned
    ns, f, c, k = _fp64_problem(n=500, seed=16)
    op, _ = _gpu_gkb(ctx, R, ns, f, c, k, 1)
    net = _constant_net(R, 17, -7.0, l_min=10, l_max=30, accept_tol=math.inf)
    st, *_ = R.make_state(torch, ns.n, 30)
    coef = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    info = learned.solve(ctx, op, _dev(f), net, st, coef)
    assert info.accepted == 1 and info.steps == 17 and math.isnan(info.eta_change)
    st2, *_ = R.make_state(torch, ns.n, 30)
    ctx.rbf_gkb(op, _dev(f), 17, st2)
    coef2 = torch.empty_like(coef)
    ctx.rbf_hkt(st2, R.RBF_FIXED_T, -7.0, coef2)
    assert torch.max(torch.abs(coef - coef2)).item() <= 1e-8 * torch.max(torch.abs(coef2)).item()


def test_learned_hkt_rejections_fall_back_to_rule(ctx, R):
    from paper_2511_09798_gb300 import learned
    ns, f, c, k = _fp64_problem(n=600, seed=15)
    nodes = _dev(ns.soa())
    lda = R.padded_lda(ns.n, R.RBF_FP64)
    A = torch.empty((ns.n, lda), dtype=torch.float64, device="cuda")
    op = ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, c, k, R.RBF_ASSEMBLED, R.RBF_FP64, A=A, lda=lda)
    ctx.rbf_assemble(op)
    st_ref, *_ = R.make_state(torch, ns.n, 40)
    ctx.rbf_gkb(op, _dev(f), 40, st_ref)
    coef_ref = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    i_ref = ctx.rbf_hkt(st_ref, R.RBF_GCV, 0.0, coef_ref)
    for net in (_constant_net(R, 20, -6.0, l_min=10, l_max=40, accept_tol=0.0),     # eta not settled
                _constant_net(R, 20, 3.0, l_min=10, l_max=40, accept_tol=1e30),      # t out of range
                _constant_net(R, 500, -6.0, l_min=10, l_max=40, accept_tol=0.0),     # clamped to l_max
                _constant_net(R, 20, -6.0, l_min=10, l_max=40, z_max=1e-3)):         # inputs out of range
        st, *_ = R.make_state(torch, ns.n, 40)
        coef = torch.empty(ns.n, dtype=torch.float64, device="cuda")
        info = learned.solve(ctx, op, _dev(f), net, st, coef)
        assert info.accepted == 0 and info.steps == 40
        assert info.l_pred in (20, 40)
        assert info.in_distribution == (0 if net.z_max == 1e-3 else 1)
        assert info.solve.index == i_ref.index
        assert torch.max(torch.abs(coef - coef_ref)).item() <= 1e-8 * torch.max(torch.abs(coef_ref)).item()
