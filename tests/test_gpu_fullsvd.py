"""GPU: full SVD by one-sided Jacobi and the full-SVD Tikhonov / TSVD
(Algorithm 3) against the FP64 oracle (LAPACK SVD through NumPy).

Tolerances: singular values are backward-stable from both sides, so they
agree to an absolute c n eps s_1 (1e-12 s_1 here).  A solution component is
f^_i phi_i / s_i, so a perturbation of the singular triplets of order
n eps s_1 moves the solution by about n eps s_1 / lambda relative (Tikhonov)
or n eps s_1 / s_k (TSVD); the tests allow 1e3 times that bound, and never
less than 1e-10.
"""
import numpy as np
import pytest

import workloads as w
from oracle import evaluate as OE
from oracle import mq as OM
from oracle import regularize as OR

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
EPS = np.finfo(float).eps


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


def _op(ctx, R, ns, c, k):
    nodes = torch.as_tensor(ns.soa(), device="cuda")
    lda = R.padded_lda(ns.n, R.RBF_FP64)
    A = torch.empty((ns.n, lda), dtype=torch.float64, device="cuda")
    op = ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, c, k, R.RBF_ASSEMBLED, R.RBF_FP64, A=A, lda=lda)
    ctx.rbf_assemble(op)
    return op


@pytest.mark.parametrize("n", [40, 41])
def test_small_svd_exact(ctx, R, n):
    rng = np.random.Generator(np.random.PCG64(50 + n))
    ns = w.NodeSet(rng.uniform(0, 1, (n, 3)), n // 2, "cube", f"rand{n}")
    op = _op(ctx, R, ns, 0.8, 1.5)
    A = OM.assemble(ns.X, ns.n_interior, 0.8, 1.5)
    f = rng.normal(size=n)
    sig = torch.empty(n, dtype=torch.float64, device="cuda")
    fh = torch.empty(n, dtype=torch.float64, device="cuda")
    V = torch.empty((n, n), dtype=torch.float64, device="cuda")  # row k = v_k
    sweeps = ctx.rbf_svd_full(op, sig, torch.as_tensor(f, device="cuda"), fh, V)
    assert 0 <= sweeps <= 40  # 0: the bidiagonalization path (n <= 1023)
    s_ref = np.linalg.svd(A, compute_uv=False)
    s = sig.cpu().numpy()
    assert np.max(np.abs(s - s_ref)) <= 1e-13 * s_ref[0]
    Vn = V.cpu().numpy().T  # columns v_k
    assert np.max(np.abs(Vn.T @ Vn - np.eye(n))) <= 1e-13
    # A v_k = sigma_k u_k and f^_k = u_k . f
    AV = A @ Vn
    assert np.max(np.abs(np.linalg.norm(AV, axis=0) - s)) <= 1e-13 * s[0]
    U = AV / s
    assert np.max(np.abs(U.T @ f - fh.cpu().numpy())) <= 1e-11 * np.linalg.norm(f) * s[0] / s[-1]


def test_cube1000_tikhonov_and_tsvd_against_oracle(ctx, R):
    ns = w.preset("cube1000")
    c, k = ns.params["c"], ns.params["k"]
    op = _op(ctx, R, ns, c, k)
    A = OM.assemble(ns.X, ns.n_interior, c, k)
    f = w.plane_wave_rhs(ns, k)
    fs = OR.full_svd(A, f)
    n = ns.n
    sig = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.rbf_svd_full(op, sig)
    assert np.max(np.abs(sig.cpu().numpy() - fs.sigma)) <= 1e-12 * fs.sigma[0]
    fd = torch.as_tensor(f, device="cuda")
    coef = torch.empty(n, dtype=torch.float64, device="cuda")
    # Tikhonov with GCV: same grid point, or an equal GCV value there
    tk = OR.tikhonov_full(A, f, "gcv", fs=fs)
    info = ctx.rbf_tikhonov(op, fd, R.RBF_GCV, 0.0, coef)
    assert info.rank == fs.r
    if info.index != tk["index"]:
        g = tk["curve"]
        assert g[info.index] <= (1 + 1e-8) * g[tk["index"]]
    # the solution at the oracle's lambda
    ctx.rbf_tikhonov(op, fd, R.RBF_FIXED, tk["lam"], coef)
    tol = max(1e-10, 1e3 * n * EPS * fs.sigma[0] / tk["lam"])
    x = coef.cpu().numpy()
    assert np.linalg.norm(x - tk["coef"]) <= tol * np.linalg.norm(tk["coef"]), tol
    P = w.test_points(ns, 500)
    u_ref = OE.reconstruct(tk["coef"], ns.X, P, c)
    u = OE.reconstruct(x, ns.X, P, c)
    assert np.max(np.abs(u - u_ref)) <= tol * np.max(np.abs(u_ref))
    # TSVD: the GCV rank, and the solution at the oracle's rank
    ts = OR.tsvd_full(A, f, fs=fs)
    it = ctx.rbf_tsvd(op, fd, 0, coef)
    if it.rank != ts["rank"]:
        cv = ts["curve"]
        assert cv[it.rank - 1] <= (1 + 1e-8) * cv[ts["rank"] - 1]
    ctx.rbf_tsvd(op, fd, ts["rank"], coef)
    tol = max(1e-10, 1e3 * n * EPS * fs.sigma[0] / fs.sigma[ts["rank"] - 1])
    assert np.linalg.norm(coef.cpu().numpy() - ts["coef"]) <= tol * np.linalg.norm(ts["coef"]), tol


@pytest.mark.parametrize("method", [0, 1])
def test_both_methods_above_1023(R, method):
    """n = 1100 by the bidiagonal path (method 0) and by one-sided Jacobi
    (method 1): singular values and the Tikhonov solution at a fixed lambda
    against the oracle."""
    ctx = R.Context(0, svd_method=method)
    n = 1100
    rng = np.random.Generator(np.random.PCG64(77))
    ns = w.cube_faces_random(n, 0.3, rng)
    op = _op(ctx, R, ns, 0.5, 2.0)
    A = OM.assemble(ns.X, ns.n_interior, 0.5, 2.0)
    f = w.plane_wave_rhs(ns, 2.0)
    fs = OR.full_svd(A, f)
    sig = torch.empty(n, dtype=torch.float64, device="cuda")
    sweeps = ctx.rbf_svd_full(op, sig)
    assert (sweeps == 0) if method == 0 else (1 <= sweeps <= 40)
    assert np.max(np.abs(sig.cpu().numpy() - fs.sigma)) <= 1e-12 * fs.sigma[0]
    lam = 1e-8 * fs.sigma[0]
    tk = OR.tikhonov_full(A, f, "fixed", lam=lam, fs=fs)
    coef = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.rbf_tikhonov(op, torch.as_tensor(f, device="cuda"), R.RBF_FIXED, lam, coef)
    tol = max(1e-10, 1e3 * n * EPS * fs.sigma[0] / lam)
    assert np.linalg.norm(coef.cpu().numpy() - tk["coef"]) <= tol * np.linalg.norm(tk["coef"])
    ctx.close()


def test_full_svd_rejects_other_operators(ctx, R):
    ns = w.cube_faces_random(200, 0.3, np.random.Generator(np.random.PCG64(3)))
    nodes = torch.as_tensor(ns.soa(), device="cuda")
    op = ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, 0.3, 2.0, R.RBF_MATRIX_FREE, R.RBF_MIXED)
    sig = torch.empty(ns.n, dtype=torch.float64, device="cuda")
    with pytest.raises(R.RbfError):
        ctx.rbf_svd_full(op, sig)
