"""GPU parity at the benchmark sizes, in the launch configurations the
benchmark times: sphere20000 (mixed, matrix-free and FP32-assembled, 150
steps), the 40 000-node casing (mixed matrix-free, learned stop and GCV-HKT)
and the 96-instance batch (833 918 rows, 150 steps).

The FP64 oracle cannot run these whole in a test, so it checks what holds at
any size (Algorithm 1 and Algorithm 4):

* the bases W_{l+1} and Z_l are orthonormal (full reorthogonalization);
* sampled rows and columns of A, computed entry by entry by the oracle, satisfy
  A Z_l = W_{l+1} C_l and A^T W_l = Z_l B_l^T (B_l the square part of C_l),
  up to the product precision, relative to s~_1;
* the projected solve and lift, recomputed by the oracle from the GPU's own
  alpha, beta and Z, give the GPU's coefficients (rel <= 1e-10), and the GPU's
  GCV choice is a minimiser of the oracle's GCV curve.

Mixed products regenerate FP32 entries (relative rounding 6e-8 per entry, FP32
partial sums): the relation residual stays below 3e-5 s~_1; a wrong sign, a
dropped term or a transposed operand moves it to about s~_1 / sqrt(N).
"""
import os

import numpy as np
import pytest

import workloads as w
from oracle import gkb as OG
from oracle import mq as OM
from oracle import regularize as OR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED_REL = 3e-5


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


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def rows_of_A(ns, c, k, idx):
    """Rows idx of the collocation matrix, entry by entry (oracle formulas)."""
    D = OM.distances(ns.X[idx], ns.X)
    out = np.empty_like(D)
    inter = np.asarray(idx) < ns.n_interior
    out[inter] = OM.lphi(D[inter], c, k)
    out[~inter] = OM.phi(D[~inter], c)
    return out


def cols_of_A(ns, c, k, idx):
    """Columns idx of the collocation matrix (N x len(idx))."""
    D = OM.distances(ns.X, ns.X[idx])
    ni = ns.n_interior
    out = np.empty_like(D)
    out[:ni] = OM.lphi(D[:ni], c, k)
    out[ni:] = OM.phi(D[ni:], c)
    return out


def sample_rows(ns, rng, n_int=32, n_bnd=16):
    ni = ns.n_interior
    a = rng.choice(ni, size=min(n_int, ni), replace=False)
    b = ni + rng.choice(ns.n - ni, size=min(n_bnd, ns.n - ni), replace=False)
    return np.sort(np.concatenate([a, b]))


def check_gkb_at_size(ns, c, k, W, Z, alpha, beta, l, rel, seed=0):
    """Orthonormality and sampled-row Golub-Kahan relations of a finished run."""
    Wl1, Zl = W[:, :l + 1], Z[:, :l]
    assert np.max(np.abs(Wl1.T @ Wl1 - np.eye(l + 1))) < 1e-12
    assert np.max(np.abs(Zl.T @ Zl - np.eye(l))) < 1e-12
    g = OG.GKBResult(W, Z, alpha, beta, l, 0, 0.0)
    C = g.C()
    s1 = np.linalg.svd(C, compute_uv=False)[0]
    idx = sample_rows(ns, np.random.default_rng(seed))
    res = rows_of_A(ns, c, k, idx) @ Zl - Wl1[idx] @ C
    assert np.max(np.abs(res)) <= rel * s1, np.max(np.abs(res)) / s1
    res_t = cols_of_A(ns, c, k, idx).T @ W[:, :l] - Zl[idx] @ C[:l].T
    assert np.max(np.abs(res_t)) <= rel * s1, np.max(np.abs(res_t)) / s1
    return g


def check_hkt_against_projected_oracle(g, lam_gpu, idx_gpu, coef_gpu, rule="gcv"):
    """The oracle's projected solve + lift on the GPU's alpha, beta, Z."""
    ps = OR.projected_svd(g.C(), g.beta1)
    if rule is not None:
        lam_or, idx_or, grid, curve = OR.choose_lambda_proj(ps, rule)
        assert idx_gpu == idx_or or curve[idx_gpu] <= curve[idx_or] * (1 + 1e-9), (idx_gpu, idx_or)
        assert lam_gpu == pytest.approx(grid[idx_gpu], rel=1e-12)
    ref = OR.hkt(g, "fixed", lam_gpu)["coef"]
    err = np.max(np.abs(coef_gpu - ref)) / np.max(np.abs(ref))
    assert err < 1e-10, err
    return ps


def gkb_arrays(st, W, Z, al, be):
    l = st.steps_done
    return (W.cpu().numpy().T.copy(), Z.cpu().numpy().T.copy(), al.cpu().numpy(), be.cpu().numpy(), l)


def test_sphere20000_mixed_both_storages(ctx, R):
    """Sphere, N = 20 000 (4000 boundary), c = 0.15, k = 10, l = 150, HKT with GCV."""
    ns = w.preset("sphere20000")
    c, k, L = 0.15, 10.0, 150
    f = dev(w.plane_wave_rhs(ns, k))
    nodes = dev(ns.soa())
    coef = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    for storage in (R.RBF_MATRIX_FREE, R.RBF_ASSEMBLED):
        A = None
        lda = 0
        if storage == R.RBF_ASSEMBLED:
            lda = R.padded_lda(ns.n, R.RBF_MIXED)
            A = torch.empty((ns.n, lda), dtype=torch.float32, device="cuda")
        op = ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, c, k, storage, R.RBF_MIXED, R.RBF_FORM_C, A, lda)
        if A is not None:
            ctx.rbf_assemble(op)
        st, W, Z, al, be = R.make_state(torch, ns.n, L)
        ctx.rbf_gkb(op, f, L, st)
        assert st.steps_done == L
        info = ctx.rbf_hkt(st, R.RBF_GCV, 0.0, coef)
        Wh, Zh, ah, bh, l = gkb_arrays(st, W, Z, al, be)
        g = check_gkb_at_size(ns, c, k, Wh, Zh, ah, bh, l, MIXED_REL, seed=int(storage))
        check_hkt_against_projected_oracle(g, info.lambda_, info.index, coef.cpu().numpy())
        del A, W, Z


def test_casing40000_learned_and_gcv(ctx, R):
    """The 40 000-node casing, c = 0.1, k = 8, Gaussian sigma = 10, mixed
    matrix-free: the learned stop with the shipped weights, then GCV-HKT(150)."""
    from paper_2511_09798_gb300 import learned
    ns = w.preset("pump40000")
    c, k, L = 0.1, 8.0, 150
    f = dev(w.gaussian_rhs(ns, 10.0, k))
    nodes = dev(ns.soa())
    op = ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, c, k, R.RBF_MATRIX_FREE, R.RBF_MIXED)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    net = learned.StopNet.load(torch, os.path.join(root, "paper_2511_09798_gb300", "stopnet_weights.npz"))
    coef = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    st, W, Z, al, be = R.make_state(torch, ns.n, L)
    li = learned.solve(ctx, op, f, net, st, coef)
    assert li.accepted == 1 and li.in_distribution == 1
    Wh, Zh, ah, bh, l = gkb_arrays(st, W, Z, al, be)
    assert l == li.steps
    g = check_gkb_at_size(ns, c, k, Wh, Zh, ah, bh, l, MIXED_REL, seed=5)
    ps = check_hkt_against_projected_oracle(g, li.solve.lambda_, -1, coef.cpu().numpy(), rule=None)
    assert li.solve.lambda_ == pytest.approx(ps.sigma[0] * 10.0 ** li.t_pred, rel=1e-10)
    # GCV-HKT(150) on the same operator
    st2, W2, Z2, al2, be2 = R.make_state(torch, ns.n, L)
    ctx.rbf_gkb(op, f, L, st2)
    info = ctx.rbf_hkt(st2, R.RBF_GCV, 0.0, coef)
    Wh, Zh, ah, bh, l = gkb_arrays(st2, W2, Z2, al2, be2)
    g2 = check_gkb_at_size(ns, c, k, Wh, Zh, ah, bh, l, MIXED_REL, seed=6)
    check_hkt_against_projected_oracle(g2, info.lambda_, info.index, coef.cpu().numpy())
    # the learned stop's first 10 steps are the same kernels on the same data
    # (after them it resumes from the stored, normalised w_11)
    assert np.array_equal(ah[:10], g.alpha[:10])


def test_batch96_full_size(ctx, R):
    """96 uneven instances (N 2000-16000), 150 steps, GCV-HKT, checked on the
    smallest, the largest and the first instance."""
    inst = w.batch_instances(96)
    L = 150
    fs = [w.plane_wave_rhs(s, s.params["k"], s.params["d"]) for s in inst]
    cs = [s.params["c"] for s in inst]
    ks = [s.params["k"] for s in inst]
    bt, keep = R.make_batch(torch, inst, cs, ks, fs, L, "cuda")
    T = int(keep["offsets"][-1])
    coef = torch.empty(T, dtype=torch.float64, device="cuda")
    ctx.rbf_batch_gkb(bt, L)
    lam = ctx.rbf_batch_hkt(bt, R.RBF_GCV, coef)
    ns_ = [s.n for s in inst]
    pick = sorted({int(np.argmin(ns_)), int(np.argmax(ns_)), 0})
    for b in pick:
        s_ = inst[b]
        n, l = s_.n, bt.steps_done[b]
        assert l == L or bt.breakdown[b] != 0
        off = int(keep["offsets"][b])
        Wb = keep["W"][(L + 1) * off:(L + 1) * off + (l + 1) * n].view(l + 1, n).cpu().numpy().T.copy()
        Zb = keep["Z"][L * off:L * off + l * n].view(l, n).cpu().numpy().T.copy()
        ab = keep["alpha"][L * b:L * b + L].cpu().numpy()
        bb = keep["beta"][(L + 1) * b:(L + 1) * (b + 1)].cpu().numpy()
        g = check_gkb_at_size(s_, cs[b], ks[b], Wb, Zb, ab, bb, l, MIXED_REL, seed=b)
        ps = OR.projected_svd(g.C(), g.beta1)
        lam_or, idx_or, grid, curve = OR.choose_lambda_proj(ps, "gcv")
        i_gpu = int(np.argmin(np.abs(grid - lam[b])))
        assert lam[b] == pytest.approx(grid[i_gpu], rel=1e-12)
        assert i_gpu == idx_or or curve[i_gpu] <= curve[idx_or] * (1 + 1e-9)
        check_hkt_against_projected_oracle(g, lam[b], i_gpu, coef[off:off + n].cpu().numpy(), rule=None)


def test_cube8000_six_solves_on_lanes(ctx, R):
    """The default benchmark's launch configuration: the six cube8000 FP64
    solves (c in {0.1, 0.2, 0.5} x k in {2, 5}, 100 steps, HKT with GCV) assembled
    and run on six concurrent lanes (rbf_gkb_many, rbf_hkt_many).  Every state and
    every coefficient vector equals the single-run path bitwise, and one solve
    is checked against the FP64 oracle directly (u at the oracle's lambda)."""
    from oracle import evaluate as OE
    ns = w.preset("cube8000")
    n, L = ns.n, 100
    cases = [(c, k) for c in (0.1, 0.2, 0.5) for k in (2.0, 5.0)]
    nodes = dev(ns.soa())
    lda = R.padded_lda(n, R.RBF_FP64)
    mats = [torch.empty((n, lda), dtype=torch.float64, device="cuda") for _ in cases]
    ops = [ctx.rbf_operator_init(nodes, n, ns.n_interior, c, k, R.RBF_ASSEMBLED, R.RBF_FP64, 0, A, lda)
           for (c, k), A in zip(cases, mats)]
    fs = {k: dev(w.plane_wave_rhs(ns, k)) for k in (2.0, 5.0)}
    bufs = [R.make_state(torch, n, L) for _ in cases]
    states = [b[0] for b in bufs]
    ctx.rbf_gkb_many(ops, [fs[k] for _, k in cases], L, states, assemble=True)
    coefs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in cases]
    infos = ctx.rbf_hkt_many(states, R.RBF_GCV, 0.0, coefs)
    for i, (c, k) in enumerate(cases):
        st1, W1, Z1, a1, b1 = R.make_state(torch, n, L)
        ctx.rbf_gkb(ops[i], fs[k], L, st1)
        assert st1.steps_done == states[i].steps_done
        _, W2, Z2, a2, b2 = bufs[i]
        assert torch.equal(a1, a2) and torch.equal(b1, b2) and torch.equal(W1, W2) and torch.equal(Z1, Z2), i
        c1 = torch.empty(n, dtype=torch.float64, device="cuda")
        inf1 = ctx.rbf_hkt(st1, R.RBF_GCV, 0.0, c1)
        assert torch.equal(c1, coefs[i]) and inf1.lambda_ == infos[i].lambda_, i
    # one of the six against the oracle: u at the oracle's GCV lambda
    i = 3
    c, k = cases[i]
    A = OM.assemble(ns.X, ns.n_interior, c, k)
    g = OG.gkb(A, None, w.plane_wave_rhs(ns, k), L)
    assert g.steps_done == states[i].steps_done
    h = OR.hkt(g, "gcv")
    coef = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.rbf_hkt(states[i], R.RBF_FIXED, h["lam"], coef)
    P = w.test_points(ns)
    u = torch.empty(P.shape[0], dtype=torch.float64, device="cuda")
    ctx.rbf_evaluate(ops[i], coef, dev(P.T), P.shape[0], u)
    u_or = OE.reconstruct(h["coef"], ns.X, P, c)
    assert np.max(np.abs(u.cpu().numpy() - u_or)) / np.max(np.abs(u_or)) < 1e-10
