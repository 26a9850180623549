"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances.  FP64 path: rel <= 1e-10 on the quantities the problem determines
(the GKB scalars up to l_stable, Ritz values >= 1e-6 s~_1, the reconstructed u
at the oracle's lambda, GCV values), tighter where the arithmetic is a single
pass (entries, products).  l_stable is the first step at which two valid FP64
reorthogonalization schemes of the oracle itself (MGS2 and CGS2) disagree by
more than 1e-12 in alpha_j or beta_{j+1}: beyond it the scalars depend on
rounding order, not on the problem.  Mixed path: products rel <= 1e-5 of
sum |A_ij x_j|, u rel <= 1e-4.
"""
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
    from paper_2511_09798_gb300 import rbfkr
    return rbfkr


@pytest.fixture(scope="module")
def ctx(R):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = R.Context(0)
    yield c
    c.close()


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def random_nodes(n, ni, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (n, 3))
    return w.NodeSet(X, ni, "cube", f"rand{n}")


def gpu_matrix(ctx, R, ns, c, k, precision=0, form=0):
    n = ns.n
    lda = R.padded_lda(n, precision)
    A = torch.full((n, lda), float("nan"), dtype=torch.float64 if precision == 0 else torch.float32, device="cuda")
    nodes = dev(ns.soa())
    op = ctx.rbf_operator_init(nodes, n, ns.n_interior, c, k, R.RBF_ASSEMBLED, precision, form, A, lda)
    ctx.rbf_assemble(op)
    return op, A[:, :n], nodes


# ---------------------------------------------------------------- assembly
@pytest.mark.parametrize("n,ni", [(1, 1), (1, 0), (7, 3), (33, 33), (33, 0), (300, 200), (1001, 617)])
def test_assembly_fp64(ctx, R, n, ni):
    ns = random_nodes(n, ni, n)
    op, A, _ = gpu_matrix(ctx, R, ns, 0.25, 3.0)
    ref = OM.assemble(ns.X, ni, 0.25, 3.0)
    got = A.cpu().numpy()
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 2e-15


@pytest.mark.parametrize("scale,c", [(1.0, 1e-3), (100.0, 0.5), (0.01, 1e-3)])
def test_assembly_fp64_wide_range(ctx, R, scale, c):
    """Entries over many decades of s = r^2 + c^2 (1e-6 .. 3e4): the refined
    FP64 reciprocal square root stays at FP64 rounding everywhere."""
    ns = random_nodes(300, 200, 11)
    ns = w.NodeSet(ns.X * scale, 200, "cube", "scaled")
    op, A, _ = gpu_matrix(ctx, R, ns, c, 3.0)
    ref = OM.assemble(ns.X, 200, c, 3.0)
    assert np.max(np.abs(A.cpu().numpy() - ref) / np.abs(ref)) < 2e-15


def test_assembly_eps_form(ctx, R):
    ns = random_nodes(200, 120, 5)
    op, A, _ = gpu_matrix(ctx, R, ns, 0.4, 2.0, form=R.RBF_FORM_EPS)
    ref = OM.assemble(ns.X, 120, 0.4, 2.0, form="eps")
    assert np.max(np.abs(A.cpu().numpy() - ref) / np.abs(ref)) < 2e-15


def test_assembly_fp32(ctx, R):
    ns = random_nodes(513, 400, 6)
    op, A, _ = gpu_matrix(ctx, R, ns, 0.1, 5.0, precision=R.RBF_MIXED)
    ref = OM.assemble(ns.X, 400, 0.1, 5.0)
    assert np.max(np.abs(A.cpu().numpy().astype(np.float64) - ref) / np.abs(ref)) < 1e-5


# ---------------------------------------------------------------- products
def _products(ctx, R, op, n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=n)
    xd = dev(x)
    y0 = torch.empty(n, dtype=torch.float64, device="cuda")
    y1 = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.rbf_matvec(op, 0, xd, y0)
    ctx.rbf_matvec(op, 1, xd, y1)
    return x, y0.cpu().numpy(), y1.cpu().numpy()


# n = 1, 2, 5: one warp takes the whole matrix; 31, 33, 95, 129: ragged 32-row
# groups and 32 / 64-column tiles; 1116, 2049: row groups and column tiles
# shared by several warps (many partial slots); 4099: ragged against every tile
@pytest.mark.parametrize("n", [1, 2, 5, 31, 33, 64, 95, 129, 257, 1003, 1116, 2049, 4099])
def test_matvec_fp64(ctx, R, n):
    ns = random_nodes(n, (2 * n) // 3, n + 1)
    op, _, _ = gpu_matrix(ctx, R, ns, 0.2, 4.0)
    A = OM.assemble(ns.X, ns.n_interior, 0.2, 4.0)
    x, y0, y1 = _products(ctx, R, op, n, 1)
    assert np.max(np.abs(y0 - A @ x) / (np.abs(A) @ np.abs(x))) < 1e-14
    assert np.max(np.abs(y1 - A.T @ x) / (np.abs(A).T @ np.abs(x))) < 1e-14


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("n", [6, 1029, 5000])
def test_matvec_mixed(ctx, R, storage, n):
    ns = random_nodes(n, (3 * n) // 4, n + 2)
    c, k = 0.15, 6.0
    if storage == 0:
        op, _, _ = gpu_matrix(ctx, R, ns, c, k, precision=R.RBF_MIXED)
    else:
        nodes = dev(ns.soa())
        op = ctx.rbf_operator_init(nodes, n, ns.n_interior, c, k, R.RBF_MATRIX_FREE, R.RBF_MIXED)
    A = OM.assemble(ns.X, ns.n_interior, c, k)
    x, y0, y1 = _products(ctx, R, op, n, 2)
    e0 = np.max(np.abs(y0 - A @ x) / (np.abs(A) @ np.abs(x)))
    e1 = np.max(np.abs(y1 - A.T @ x) / (np.abs(A).T @ np.abs(x)))
    # the measured error of the FP32 products against the FP64 oracle, recorded
    print(f"mixed product storage={storage} n={n}: max |y - y_or| / (|A||x|) = {e0:.2e} (A x), {e1:.2e} (A^T x); "
          f"|y - y_or| / |y_or| = {np.linalg.norm(y0 - A @ x) / np.linalg.norm(A @ x):.2e}, "
          f"{np.linalg.norm(y1 - A.T @ x) / np.linalg.norm(A.T @ x):.2e}")
    assert e0 < 1e-5 and e1 < 1e-5


# The FP32 matrix-free products run over tile pairs (blocks of 128 nodes, of
# 256 from about 8700 nodes on): n_interior at 0, n, inside a 32-column group,
# on a group edge and on a block edge; n = 1, below one group, ragged last
# blocks; 9001 takes the 256 blocks.
@pytest.mark.parametrize("n,ni", [(1, 0), (1, 1), (5, 3), (31, 31), (33, 0), (128, 100), (129, 128), (300, 160),
                                  (300, 161), (1000, 1000), (2500, 1777), (9001, 6000)])
def test_matvec_mixed_matrix_free_tile_pairs(ctx, R, n, ni):
    ns = random_nodes(n, ni, n + 7)
    c, k = 0.2, 5.0
    op = ctx.rbf_operator_init(dev(ns.soa()), n, ni, c, k, R.RBF_MATRIX_FREE, R.RBF_MIXED)
    A = OM.assemble(ns.X, ni, c, k)
    x, y0, y1 = _products(ctx, R, op, n, 3)
    e0 = np.max(np.abs(y0 - A @ x) / (np.abs(A) @ np.abs(x)))
    e1 = np.max(np.abs(y1 - A.T @ x) / (np.abs(A).T @ np.abs(x)))
    print(f"matrix-free FP32 n={n} ni={ni}: {e0:.2e} (A x), {e1:.2e} (A^T x) of |A||x|")
    assert e0 < 1e-5 and e1 < 1e-5
    _, z0, z1 = _products(ctx, R, op, n, 3)  # same input: bitwise the same result
    assert np.array_equal(z0, y0) and np.array_equal(z1, y1)


@pytest.mark.parametrize("n", [300, 5000])
def test_mixed_matrix_free_eps_form(ctx, R, n):
    """The eps form scales every entry by 1/c: the FP32 slots are unscaled runs
    and the consumers (the matvec's reduction, the GKB half-step) apply 1/c.
    Products against the dense eps-form oracle matrix, and the first GKB
    scalars against the oracle's run (FP32 entries: rel <= 1e-5)."""
    ns = random_nodes(n, (2 * n) // 3, n + 9)
    c, k = 0.3, 3.0
    op = ctx.rbf_operator_init(dev(ns.soa()), n, ns.n_interior, c, k, R.RBF_MATRIX_FREE, R.RBF_MIXED,
                               R.RBF_FORM_EPS)
    A = OM.assemble(ns.X, ns.n_interior, c, k, form="eps")
    x, y0, y1 = _products(ctx, R, op, n, 8)
    assert np.max(np.abs(y0 - A @ x) / (np.abs(A) @ np.abs(x))) < 1e-5
    assert np.max(np.abs(y1 - A.T @ x) / (np.abs(A).T @ np.abs(x))) < 1e-5
    f = w.plane_wave_rhs(ns, k)
    g = OG.gkb(A, None, f, 6)
    st, _, _, al, be = run_gkb(ctx, R, op, f, 6, n)
    assert st.steps_done == 6
    assert np.max(np.abs(al[:4] - g.alpha[:4]) / g.alpha[:4]) < 1e-5
    assert np.max(np.abs(be[1:5] - g.beta[1:5]) / g.beta[1:5]) < 1e-5


def test_matvec_mixed_matrix_free_folded_slots(ctx, R):
    """26 000 nodes: 102 blocks of 256, more partial slots than the half-step
    stages (71 at 172 rows per SM), folded in pairs before it.  Checked on
    sampled rows of A x and columns of A^T x (block edges, n_interior, both
    ends)."""
    n, ni, c, k = 26000, 20000, 0.1, 8.0
    ns = random_nodes(n, ni, 26)
    op = ctx.rbf_operator_init(dev(ns.soa()), n, ni, c, k, R.RBF_MATRIX_FREE, R.RBF_MIXED)
    x, y0, y1 = _products(ctx, R, op, n, 4)
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([[0, 1, 255, 256, 257, ni - 1, ni, ni + 1, n - 2, n - 1],
                                    rng.integers(0, n, 150)]))
    interior = np.arange(n) < ni
    D = OM.distances(ns.X[idx], ns.X)  # rows idx of A
    Ar = np.where(interior[idx, None], OM.lphi(D, c, k), OM.phi(D, c))
    e0 = np.max(np.abs(y0[idx] - Ar @ x) / (np.abs(Ar) @ np.abs(x)))
    Ac = np.where(interior[:, None], OM.lphi(D.T, c, k), OM.phi(D.T, c))  # columns idx of A
    e1 = np.max(np.abs(y1[idx] - Ac.T @ x) / (np.abs(Ac).T @ np.abs(x)))
    print(f"matrix-free FP32 n={n}: {e0:.2e} (A x), {e1:.2e} (A^T x) of |A||x| on {idx.size} samples")
    assert e0 < 1e-5 and e1 < 1e-5


# FP64 matrix-free products by tile pairs of 128-node blocks: the same edge
# cases as the FP32 tile pairs (n_interior at 0, n, inside a 32-column group,
# on group and block edges; n = 1; ragged last blocks).
@pytest.mark.parametrize("n,ni", [(1, 0), (1, 1), (6, 4), (31, 31), (33, 0), (128, 100), (129, 128), (300, 160),
                                  (300, 161), (1029, 771), (5000, 3750)])
def test_matvec_fp64_matrix_free(ctx, R, n, ni):
    """FP64 operators regenerate the entries in FP64 (matrix-free): products
    agree with the dense FP64 matrix to rounding, bitwise the same on a rerun."""
    ns = random_nodes(n, ni, n + 5)
    c, k = 0.25, 3.0
    op = ctx.rbf_operator_init(dev(ns.soa()), n, ni, c, k, R.RBF_MATRIX_FREE, R.RBF_FP64)
    A = OM.assemble(ns.X, ni, c, k)
    x, y0, y1 = _products(ctx, R, op, n, 3)
    assert np.max(np.abs(y0 - A @ x) / (np.abs(A) @ np.abs(x))) < 1e-13
    assert np.max(np.abs(y1 - A.T @ x) / (np.abs(A).T @ np.abs(x))) < 1e-13
    _, z0, z1 = _products(ctx, R, op, n, 3)
    assert np.array_equal(z0, y0) and np.array_equal(z1, y1)


def test_gkb_fp64_matrix_free_matches_assembled(ctx, R):
    ns = random_nodes(900, 640, 77)
    c, k = 0.3, 2.0
    f = w.plane_wave_rhs(ns, k)
    op_a, _, _ = gpu_matrix(ctx, R, ns, c, k)
    op_m = ctx.rbf_operator_init(dev(ns.soa()), ns.n, ns.n_interior, c, k, R.RBF_MATRIX_FREE, R.RBF_FP64)
    A = OM.assemble(ns.X, ns.n_interior, c, k)
    ls = max(1, l_stable(A, f, 30)[0])
    st_a, _, _, al_a, be_a = run_gkb(ctx, R, op_a, f, 30, ns.n)
    st_m, _, _, al_m, be_m = run_gkb(ctx, R, op_m, f, 30, ns.n)
    assert st_a.steps_done == st_m.steps_done
    assert np.max(np.abs(al_m[:ls] - al_a[:ls]) / al_a[:ls]) < 1e-10
    assert np.max(np.abs(be_m[1:ls + 1] - be_a[1:ls + 1]) / be_a[1:ls + 1]) < 1e-10
    ca = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    cm = torch.empty_like(ca)
    ia = ctx.rbf_hkt(st_a, R.RBF_FIXED_T, -6.0, ca)
    ctx.rbf_hkt(st_m, R.RBF_FIXED_T, -6.0, cm)
    assert torch.max(torch.abs(ca - cm)).item() <= 1e-8 * torch.max(torch.abs(ca)).item(), ia.lambda_


# ---------------------------------------------------------------- GKB
def run_gkb(ctx, R, op, f, steps, n):
    st, W, Z, al, be = R.make_state(torch, n, steps)
    ctx.rbf_gkb(op, dev(f), steps, st)
    return st, W.cpu().numpy().T, Z.cpu().numpy().T, al.cpu().numpy(), be.cpu().numpy()


def l_stable(A, f, steps):
    g1 = OG.gkb(A, None, f, steps, reorth="mgs2")
    g2 = OG.gkb(A, None, f, steps, reorth="cgs2")
    l = min(g1.steps_done, g2.steps_done)
    rel = np.maximum(np.abs(g1.alpha[:l] - g2.alpha[:l]) / g1.alpha[:l],
                     np.abs(g1.beta[1:l + 1] - g2.beta[1:l + 1]) / np.maximum(g1.beta[1:l + 1], 1e-300))
    bad = np.flatnonzero(rel > 1e-12)
    return (int(bad[0]) if len(bad) else l), g1


@pytest.mark.parametrize("n,ni,steps", [(400, 260, 50), (1001, 700, 80), (97, 60, 97)])
def test_gkb_fp64_parity(ctx, R, n, ni, steps):
    ns = random_nodes(n, ni, 3 * n)
    c, k = 0.2, 3.0
    op, _, _ = gpu_matrix(ctx, R, ns, c, k)
    A = OM.assemble(ns.X, ni, c, k)
    f = np.random.default_rng(n).normal(size=n)
    ls, g = l_stable(A, f, steps)
    st, W, Z, al, be = run_gkb(ctx, R, op, f, steps, n)
    assert st.steps_done == g.steps_done and st.breakdown == g.breakdown
    m = max(1, ls)
    print(f"GKB scalars compared to rel 1e-10 for j <= l_stable = {ls} of {g.steps_done} steps (n = {n})")
    assert np.max(np.abs(al[:m] - g.alpha[:m]) / g.alpha[:m]) < 1e-10
    assert np.max(np.abs(be[:m + 1] - g.beta[:m + 1]) / g.beta[:m + 1]) < 1e-10
    # Algorithm 1 relations hold for the GPU's own bases
    l = st.steps_done
    C = np.zeros((l + 1, l))
    C[np.arange(l), np.arange(l)] = al[:l]
    C[np.arange(1, l + 1), np.arange(l)] = be[1:l + 1]
    nA = np.linalg.norm(A)
    assert np.linalg.norm(A @ Z[:, :l] - W[:, :l + 1] @ C) / nA < 1e-12
    assert np.linalg.norm(A.T @ W[:, :l] - Z[:, :l] @ C[:l].T) / nA < 1e-12
    Wl = W[:, :l + 1] if st.breakdown != 2 else W[:, :l]  # w_{l+1} = 0 after a beta breakdown
    assert np.max(np.abs(Wl.T @ Wl - np.eye(Wl.shape[1]))) < 1e-12
    assert np.max(np.abs(Z[:, :l].T @ Z[:, :l] - np.eye(l))) < 1e-12


def test_gkb_deterministic_and_resume(ctx, R):
    n = 777
    ns = random_nodes(n, 500, 9)
    op, _, _ = gpu_matrix(ctx, R, ns, 0.3, 2.0)
    f = np.random.default_rng(1).normal(size=n)
    _, W1, Z1, a1, b1 = run_gkb(ctx, R, op, f, 30, n)
    _, W2, Z2, a2, b2 = run_gkb(ctx, R, op, f, 30, n)
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2) and np.array_equal(W1, W2)
    st, W, Z, al, be = R.make_state(torch, n, 30)
    ctx.rbf_gkb(op, dev(f), 12, st)
    ctx.rbf_gkb_resume(op, st, 18)
    assert st.steps_done == 30
    # the resumed run restarts from the stored normalised w_13 rather than the raw
    # vector, so it agrees to rounding, not bit for bit
    assert np.max(np.abs(al.cpu().numpy() - a1) / a1) < 1e-10
    assert np.max(np.abs(be.cpu().numpy() - b1) / b1) < 1e-10
    assert np.max(np.abs(Z.cpu().numpy().T - Z1)) < 1e-9


def test_gkb_host_snapshot_restore_resume(ctx, R):
    """A run checkpointed to host memory after 12 steps, restored into fresh
    buffers on another context and resumed gives the bits of the same run
    resumed in place."""
    n = 777
    ns = random_nodes(n, 500, 9)
    op, _, _ = gpu_matrix(ctx, R, ns, 0.3, 2.0)
    f = np.random.default_rng(1).normal(size=n)
    st, W, Z, al, be = R.make_state(torch, n, 30)
    ctx.rbf_gkb(op, dev(f), 12, st)
    snap = ctx.rbf_gkb_snapshot(st)
    assert snap["steps_done"] == 12 and np.array_equal(snap["alpha"], al[:12].cpu().numpy())
    assert np.array_equal(snap["W"], W[:13].cpu().numpy()) and np.array_equal(snap["Z"], Z[:12].cpu().numpy())
    ctx.rbf_gkb_resume(op, st, 18)
    ctx2 = R.Context(0)
    st2, W2, Z2, al2, be2 = R.make_state(torch, n, 30)
    ctx2.rbf_gkb_restore(st2, snap)
    assert (st2.steps_done, st2.breakdown, st2.c_hat) == (12, snap["breakdown"], snap["c_hat"])
    ctx2.rbf_gkb_resume(op, st2, 18)
    torch.cuda.synchronize()
    assert st2.steps_done == st.steps_done == 30
    assert torch.equal(al2, al) and torch.equal(be2, be) and torch.equal(W2, W) and torch.equal(Z2, Z)
    with pytest.raises(R.RbfError):  # more steps than the buffers hold
        st3 = R.make_state(torch, n, 8)[0]
        ctx2.rbf_gkb_restore(st3, snap)
    ctx2.close()


def _write_matrix(ctx, R, A):
    n = A.shape[0]
    lda = R.padded_lda(n, 0)
    Ad = torch.zeros((n, lda), dtype=torch.float64, device="cuda")
    Ad[:, :n] = dev(A)
    nodes = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    op = ctx.rbf_operator_init(nodes, n, n, 1.0, 0.0, R.RBF_ASSEMBLED, R.RBF_FP64, 0, Ad, lda)
    op._keep2 = Ad
    return op


def test_breakdown_beta_on_rank_deficient(ctx, R):
    rng = np.random.default_rng(2)
    n, r = 60, 12
    U, _ = np.linalg.qr(rng.normal(size=(n, r)))
    V, _ = np.linalg.qr(rng.normal(size=(n, r)))
    A = U @ np.diag(np.logspace(0, -3, r)) @ V.T
    f = A @ rng.normal(size=n)
    op = _write_matrix(ctx, R, A)
    st, W, Z, al, be = run_gkb(ctx, R, op, f, 30, n)
    g = OG.gkb(A, None, f, 30)
    assert (st.steps_done, st.breakdown) == (g.steps_done, g.breakdown) == (r, 2)
    assert be[r] == 0.0 and np.all(W[:, r] == 0.0)
    coef = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.rbf_hkt(st, R.RBF_FIXED, 1e-14, coef)
    x_min = np.linalg.pinv(A) @ f
    assert np.linalg.norm(coef.cpu().numpy() - x_min) / np.linalg.norm(x_min) < 1e-8


def test_breakdown_alpha_first_step(ctx, R):
    rng = np.random.default_rng(3)
    n = 30
    A = rng.normal(size=(n, n))
    A[20:] = 0.0
    f = np.zeros(n)
    f[25] = 1.0
    op = _write_matrix(ctx, R, A)
    st, *_ = run_gkb(ctx, R, op, f, 10, n)
    assert st.steps_done == 0 and st.breakdown == 1


def test_zero_rhs(ctx, R):
    op = _write_matrix(ctx, R, np.eye(8))
    st, *_ = run_gkb(ctx, R, op, np.zeros(8), 3, 8)
    assert st.steps_done == 0 and st.breakdown == 1


# ---------------------------------------------------------------- projected problem
def gpu_projected(ctx, R, st, l):
    sig = torch.empty(l, dtype=torch.float64, device="cuda")
    ft = torch.empty(l + 1, dtype=torch.float64, device="cuda")
    V = torch.empty((l, l), dtype=torch.float64, device="cuda")
    ctx.rbf_projected_svd(st, sig, ft, V, l)
    return sig.cpu().numpy(), ft.cpu().numpy(), V.cpu().numpy().T  # V[:, i] = v_i


def _check_projected(ps, sig, ft, V, beta1):
    l = ps.l
    s1 = ps.sigma[0]
    keep = ps.sigma >= 1e-6 * s1
    assert np.all(np.abs(sig[keep] - ps.sigma[keep]) <= 1e-10 * ps.sigma[keep] + 1e-13 * s1)
    assert np.allclose(np.sort(sig)[::-1], sig)
    assert np.max(np.abs(V.T @ V - np.eye(l))) < 1e-10
    assert abs(np.sum(ft ** 2) - beta1 ** 2) / beta1 ** 2 < 1e-12
    for t in (-12, -8, -4, -1):
        lam = s1 * 10.0 ** t
        y_or = OR.hkt_solve_proj(ps, lam)
        y = V @ (sig * ft[:l] / (sig ** 2 + lam ** 2))
        assert np.linalg.norm(y - y_or) / np.linalg.norm(y_or) < 1e-10, t


def test_projected_svd_random_mq(ctx, R):
    n = 600
    ns = random_nodes(n, 400, 11)
    op, _, _ = gpu_matrix(ctx, R, ns, 0.25, 3.0)
    A = OM.assemble(ns.X, 400, 0.25, 3.0)
    f = np.random.default_rng(5).normal(size=n)
    st, W, Z, al, be = run_gkb(ctx, R, op, f, 60, n)
    g = OG.GKBResult(W, Z, al, be, st.steps_done, st.breakdown, st.c_hat)
    ps = OR.projected_svd(g.C(), g.beta1)  # oracle SVD of the GPU's own C
    sig, ft, V = gpu_projected(ctx, R, st, st.steps_done)
    _check_projected(ps, sig, ft, V, g.beta1)


def test_projected_svd_clusters_cube_grid(ctx, R):
    # the symmetric grid gives (near-)repeated Ritz values
    ns = w.cube_grid(10)
    op, _, _ = gpu_matrix(ctx, R, ns, 0.3, 2.0)
    f = w.plane_wave_rhs(ns, 2.0)
    st, W, Z, al, be = run_gkb(ctx, R, op, f, 40, ns.n)
    g = OG.GKBResult(W, Z, al, be, st.steps_done, st.breakdown, st.c_hat)
    ps = OR.projected_svd(g.C(), g.beta1)
    sig, ft, V = gpu_projected(ctx, R, st, st.steps_done)
    _check_projected(ps, sig, ft, V, g.beta1)


@pytest.mark.parametrize("l", [1, 2, 3, 17])
def test_projected_svd_tiny(ctx, R, l):
    rng = np.random.default_rng(l)
    n = 40
    A = rng.normal(size=(n, n))
    f = rng.normal(size=n)
    op = _write_matrix(ctx, R, A)
    st, W, Z, al, be = run_gkb(ctx, R, op, f, l, n)
    g = OG.GKBResult(W, Z, al, be, st.steps_done, st.breakdown, st.c_hat)
    ps = OR.projected_svd(g.C(), g.beta1)
    sig, ft, V = gpu_projected(ctx, R, st, l)
    _check_projected(ps, sig, ft, V, g.beta1)


# ---------------------------------------------------------------- methods
def _solve_case(ctx, R, ns, c, k, steps, f=None):
    op, _, _ = gpu_matrix(ctx, R, ns, c, k)
    A = OM.assemble(ns.X, ns.n_interior, c, k)
    f = w.plane_wave_rhs(ns, k) if f is None else f
    st, W, Z, al, be = R.make_state(torch, ns.n, steps)
    ctx.rbf_gkb(op, dev(f), steps, st)
    g = OG.gkb(A, None, f, steps)
    return op, st, g, A, f


@pytest.mark.parametrize("rule", ["gcv", "lcurve"])
def test_hkt_parity(ctx, R, rule):
    ns = w.cube_faces_random(800, 0.35, np.random.Generator(np.random.PCG64(4)))
    c, k, steps = 0.25, 3.0, 60
    op, st, g, A, f = _solve_case(ctx, R, ns, c, k, steps)
    P = w.test_points(ns, 500)
    Pd = dev(P.T)
    coef = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    u = torch.empty(500, dtype=torch.float64, device="cuda")
    curve = torch.empty(321, dtype=torch.float64, device="cuda")
    rc = R.RBF_GCV if rule == "gcv" else R.RBF_LCURVE
    info = ctx.rbf_hkt(st, rc, 0.0, coef, curve)
    h = OR.hkt(g, rule)
    ps = h["ps"]
    if info.index != h["index"]:
        if rule == "gcv":
            gv = OR.gcv_proj(ps, np.array([info.lambda_, h["lam"]]))
            assert gv[0] <= (1 + 1e-10) * gv[1]
        else:
            # a flat curvature maximum: the GPU's corner must be a maximum of the
            # oracle's curvature to within its rounding (second differences / h^2)
            kap = h["curve"]
            assert kap[info.index - 1] >= kap[h["index"] - 1] - 1e-6 * abs(kap[h["index"] - 1])
    else:
        assert info.lambda_ == pytest.approx(h["lam"], rel=1e-13)
    if rule == "gcv":
        cg = curve.cpu().numpy()
        assert np.allclose(cg, h["curve"], rtol=1e-9, atol=0)
    # u at the oracle's lambda
    ctx.rbf_hkt(st, R.RBF_FIXED, h["lam"], coef)
    ctx.rbf_evaluate(op, coef, Pd, 500, u)
    u_or = OE.reconstruct(h["coef"], ns.X, P, c)
    assert np.max(np.abs(u.cpu().numpy() - u_or)) / np.max(np.abs(u_or)) < 1e-10


def test_ine_tsvd_parity(ctx, R):
    ns = w.cube_faces_random(700, 0.35, np.random.Generator(np.random.PCG64(8)))
    c, k, steps = 0.3, 2.0, 50
    op, st, g, A, f = _solve_case(ctx, R, ns, c, k, steps)
    P = w.test_points(ns, 300)
    coef = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    u = torch.empty(300, dtype=torch.float64, device="cuda")
    info = ctx.rbf_ine_tsvd(st, 0, coef)
    t = OR.ine_tsvd(g)
    assert info.rank == t["rank"]
    for rank in (t["rank"], 5, 20):
        ctx.rbf_ine_tsvd(st, rank, coef)
        ctx.rbf_evaluate(op, coef, dev(P.T), 300, u)
        u_or = OE.reconstruct(OR.ine_tsvd(g, rank=rank)["coef"], ns.X, P, c)
        assert np.max(np.abs(u.cpu().numpy() - u_or)) / np.max(np.abs(u_or)) < 1e-10


def test_evaluate_fp64(ctx, R):
    ns = random_nodes(1500, 900, 21)
    nodes = dev(ns.soa())
    op = ctx.rbf_operator_init(nodes, ns.n, 900, 0.2, 1.0, R.RBF_MATRIX_FREE, R.RBF_MIXED)
    coef = np.random.default_rng(0).normal(size=ns.n)
    P = np.random.default_rng(1).uniform(0, 1, (333, 3))
    u = torch.empty(333, dtype=torch.float64, device="cuda")
    ctx.rbf_evaluate(op, dev(coef), dev(P.T), 333, u)
    ref = OE.reconstruct(coef, ns.X, P, 0.2)
    scale = OM.phi(OM.distances(P, ns.X), 0.2) @ np.abs(coef)
    assert np.max(np.abs(u.cpu().numpy() - ref) / scale) < 1e-14


# ---------------------------------------------------------------- workloads at size
def test_cube1000_workload(ctx, R):
    """Symmetric 10^3 grid (c = 0.3, k = 2, l = 40): tolerances from the oracle's own spread."""
    ns = w.cube_grid(10)
    c, k, steps = 0.3, 2.0, 40
    op, st, g, A, f = _solve_case(ctx, R, ns, c, k, steps)
    ls, _ = l_stable(A, f, steps)
    al = np.empty(steps)
    assert st.steps_done == g.steps_done
    g2 = OG.gkb(A, None, f, steps, reorth="cgs2")
    P = w.test_points(ns)
    coef = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    u = torch.empty(P.shape[0], dtype=torch.float64, device="cuda")
    for rule in ("gcv", "lcurve"):
        h = OR.hkt(g, rule)
        ctx.rbf_hkt(st, R.RBF_FIXED, h["lam"], coef)
        ctx.rbf_evaluate(op, coef, dev(P.T), P.shape[0], u)
        u_or = OE.reconstruct(h["coef"], ns.X, P, c)
        u_or2 = OE.reconstruct(OR.hkt(g2, "fixed", h["lam"])["coef"], ns.X, P, c)
        spread = np.max(np.abs(u_or2 - u_or)) / np.max(np.abs(u_or))
        err = np.max(np.abs(u.cpu().numpy() - u_or)) / np.max(np.abs(u_or))
        assert err <= max(1e-10, 10 * spread), (rule, err, spread)


@pytest.mark.slow
def test_cube8000_fp64_parity(ctx, R):
    """N = 8000 Halton cube, l = 100 (the benchmark configuration), FP64 assembled."""
    ns = w.preset("cube8000")
    c, k, steps = 0.2, 5.0, 100
    op, st, g, A, f = _solve_case(ctx, R, ns, c, k, steps)
    assert st.steps_done == g.steps_done
    ls, _ = l_stable(A, f, steps)
    al = np.empty(0)
    st2, W, Z, al, be = run_gkb(ctx, R, op, f, steps, ns.n)
    m = max(1, ls)
    print(f"cube8000: GKB scalars compared to rel 1e-10 for j <= l_stable = {ls} of {steps} steps")
    assert np.max(np.abs(al[:m] - g.alpha[:m]) / g.alpha[:m]) < 1e-10
    P = w.test_points(ns)
    coef = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    u = torch.empty(P.shape[0], dtype=torch.float64, device="cuda")
    for rule in ("gcv", "lcurve"):
        h = OR.hkt(g, rule)
        ctx.rbf_hkt(st2, R.RBF_FIXED, h["lam"], coef)
        ctx.rbf_evaluate(op, coef, dev(P.T), P.shape[0], u)
        u_or = OE.reconstruct(h["coef"], ns.X, P, c)
        assert np.max(np.abs(u.cpu().numpy() - u_or)) / np.max(np.abs(u_or)) < 1e-10


def test_mixed_matrix_free_solution(ctx, R):
    """Mixed precision (FP32 regenerated entries) against the FP64 oracle: u rel <= 1e-4."""
    ns = w.sphere_fibonacci_ball(600, 2400, seed=3)
    c, k, steps = 0.15, 4.0, 150
    A = OM.assemble(ns.X, ns.n_interior, c, k)
    f = w.plane_wave_rhs(ns, k)
    g = OG.gkb(A, None, f, steps)
    P = w.test_points(ns, 400)
    nodes = dev(ns.soa())
    coef = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    u = torch.empty(400, dtype=torch.float64, device="cuda")
    for storage in (R.RBF_MATRIX_FREE, R.RBF_ASSEMBLED):
        if storage == R.RBF_ASSEMBLED:
            op, _, _ = gpu_matrix(ctx, R, ns, c, k, precision=R.RBF_MIXED)
        else:
            op = ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, c, k, storage, R.RBF_MIXED)
        st, *_ = R.make_state(torch, ns.n, steps)
        ctx.rbf_gkb(op, dev(f), steps, st)
        for rule in ("gcv", "lcurve"):
            h = OR.hkt(g, rule)
            ctx.rbf_hkt(st, R.RBF_FIXED, h["lam"], coef)
            ctx.rbf_evaluate(op, coef, dev(P.T), 400, u)
            u_or = OE.reconstruct(h["coef"], ns.X, P, c)
            err = np.max(np.abs(u.cpu().numpy() - u_or)) / np.max(np.abs(u_or))
            print(f"mixed storage={storage} rule={rule} lambda/s1={h['lam'] / h['ps'].sigma[0]:.2e} "
                  f"max|u|={np.max(np.abs(u_or)):.3f} rel={err:.2e}")
            assert err < 1e-4


def test_invalid_arguments(ctx, R):
    nodes = torch.zeros((3, 10), dtype=torch.float64, device="cuda")
    for args in [(nodes, 0, 0, 0.1, 1.0), (nodes, 10, 11, 0.1, 1.0), (nodes, 10, 5, 0.0, 1.0),
                 (nodes, 10, 5, 0.1, -1.0)]:
        with pytest.raises(R.RbfError) as e:
            ctx.rbf_operator_init(*args, R.RBF_MATRIX_FREE, R.RBF_MIXED)
        assert e.value.status == R.RBF_ERR_INVALID
    with pytest.raises(R.RbfError) as e:  # assembled without a matrix
        ctx.rbf_operator_init(nodes, 10, 5, 0.1, 1.0, R.RBF_ASSEMBLED, R.RBF_FP64)
    assert e.value.status == R.RBF_ERR_INVALID
    op = ctx.rbf_operator_init(nodes, 10, 5, 0.1, 1.0, R.RBF_MATRIX_FREE, R.RBF_MIXED)
    st, *_ = R.make_state(torch, 10, 4)
    with pytest.raises(R.RbfError) as e:
        ctx.rbf_gkb(op, torch.zeros(10, dtype=torch.float64, device="cuda"), 5, st)
    assert e.value.status == R.RBF_ERR_INVALID
    with pytest.raises(R.RbfError) as e:
        ctx.rbf_tikhonov(op, torch.zeros(10, dtype=torch.float64, device="cuda"), 0, 0.0,
                         torch.zeros(10, dtype=torch.float64, device="cuda"))
    assert e.value.status == R.RBF_ERR_UNSUPPORTED
