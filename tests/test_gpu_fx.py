"""GPU: the FP64 assembled GKB products in exact integer fixed point.

For FP64 assembled operators (n <= 16384) GKB computes A z and A^T w from
int64 fixed-point copies of A (k_gemv_flat_fx, k_gemv_t_fx) unless the
context sets fma_products.  The first GKB step holds one product of each kind:
alpha_1 z_1 = A^T f / beta_1 and beta_2 w_2 = A z_1 - alpha_1 w_1 (Algorithm 1;
at j = 1 the reorthogonalization removes only rounding-level components).
They are compared with exact sums (Python integers) over the matrix the GPU
holds, on sampled rows and columns, at 1e-14 of sum |A_ij x_j| plus the
normwise bound of the fixed-point roundings, 2^-60 (max|A| |x|_1 + |A|_1
max|x|) per output.  A planted mistake in the arithmetic (a dropped limb
product: ~2^-21 relative; a wrong scale; a wrong column) fails these by
orders of magnitude.  The GKB run with the fixed-point products is also
compared with the run with FP64 FMA products.
"""
from fractions import Fraction

import numpy as np
import pytest

import workloads as w
from oracle import gkb as OG
from oracle import mq as OM

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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def exact_dot(a, x):
    """sum_j a_j x_j exactly, as (numerator integer, power of two)."""
    ma, ea = np.frexp(np.asarray(a, dtype=np.float64))
    mx, ex = np.frexp(np.asarray(x, dtype=np.float64))
    ia = (ma * 2.0 ** 53).astype(np.int64)
    ix = (mx * 2.0 ** 53).astype(np.int64)
    e = (ea.astype(np.int64) + ex.astype(np.int64) - 106)
    nz = (ia != 0) & (ix != 0)
    if not nz.any():
        return 0, 0
    emin = int(e[nz].min())
    tot = 0
    for p, q, k in zip(ia[nz].tolist(), ix[nz].tolist(), e[nz].tolist()):
        tot += (p * q) << (k - emin)
    return tot, emin


def to_float(num, e2, minus=0.0):
    """num 2^e2 - minus, exactly, then rounded once to FP64."""
    return float(Fraction(num) * Fraction(2) ** e2 - Fraction(minus))


def check_first_step(ctx, R, A_gpu, op, f, label, samples=24, seed=0):
    """Both products of step 1 against exact sums on sampled rows / columns."""
    n = A_gpu.shape[0]
    st, W, Z, al, be = R.make_state(torch, n, 1)
    ctx.rbf_gkb(op, dev(f), 1, st)
    W, Z = W.cpu().numpy().T, Z.cpu().numpy().T
    al, be = al.cpu().numpy(), be.cpu().numpy()
    A = A_gpu
    rng = np.random.default_rng(seed)
    idx = np.arange(n) if n <= samples else np.sort(rng.choice(n, samples, replace=False))
    b1, a1 = be[0], al[0]
    assert st.breakdown in (0, 2) and np.isfinite(b1) and np.isfinite(a1), (label, st.breakdown)
    worst = 0.0
    # r-side: alpha_1 z_1 = A^T f / beta_1
    for j in idx:
        num, e2 = exact_dot(A[:, j], f)
        ref = to_float(num, e2) / b1
        got = a1 * Z[j, 0]
        absum = np.sum(np.abs(A[:, j] * f)) / b1
        bound = 1e-14 * absum + 2.0 ** -60 * (np.max(np.abs(A[:, j])) * np.sum(np.abs(f))
                                               + np.sum(np.abs(A[:, j])) * np.max(np.abs(f))) / b1
        worst = max(worst, abs(got - ref) / max(absum, 1e-300))
        assert abs(got - ref) <= bound, (label, "A^T", j, got, ref, absum)
    if st.breakdown != 0:
        return worst
    # p-side: beta_2 w_2 = A z_1 - alpha_1 w_1 (w_1 = f / beta_1 as stored)
    z1, w1, b2 = Z[:, 0], W[:, 0], be[1]
    for i in idx:
        num, e2 = exact_dot(A[i, :], z1)
        ref = to_float(num, e2, a1 * w1[i])
        got = b2 * W[i, 1]
        absum = np.sum(np.abs(A[i, :] * z1)) + abs(a1 * w1[i])
        bound = 1e-14 * absum + 2.0 ** -60 * (np.max(np.abs(A[i, :])) * np.sum(np.abs(z1))
                                               + np.sum(np.abs(A[i, :])) * np.max(np.abs(z1)))
        worst = max(worst, abs(got - ref) / max(absum, 1e-300))
        assert abs(got - ref) <= bound, (label, "A", i, got, ref, absum)
    return worst


def random_nodes(n, ni, seed):
    rng = np.random.default_rng(seed)
    return w.NodeSet(rng.uniform(0, 1, (n, 3)), ni, "cube", f"rand{n}")


def gpu_operator(ctx, R, ns, c, k):
    n = ns.n
    lda = R.padded_lda(n, R.RBF_FP64)
    A = torch.full((n, lda), float("nan"), dtype=torch.float64, device="cuda")
    nodes = dev(ns.soa())
    op = ctx.rbf_operator_init(nodes, n, ns.n_interior, c, k, R.RBF_ASSEMBLED, R.RBF_FP64, R.RBF_FORM_C, A, lda)
    ctx.rbf_assemble(op)
    op._keep_fx = (A, nodes)
    return op, A[:, :n].cpu().numpy()


@pytest.mark.parametrize("n,ni", [(1, 1), (2, 1), (5, 3), (33, 20), (129, 128), (1003, 700), (2049, 1500),
                                  (4099, 3000), (9001, 6000)])
def test_fx_products_exact_sums(ctx, R, n, ni):
    ns = random_nodes(n, ni, 11 * n)
    op, A = gpu_operator(ctx, R, ns, 0.3, 4.0)
    f = np.random.default_rng(n + 1).normal(size=n)
    worst = check_first_step(ctx, R, A, op, f, f"n={n}")
    print(f"n = {n}: worst |error| / sum|A x| = {worst:.2e}")


def _write_matrix(ctx, R, A):
    n = A.shape[0]
    lda = R.padded_lda(n, R.RBF_FP64)
    Ad = torch.zeros((n, lda), dtype=torch.float64, device="cuda")
    Ad[:, :n] = dev(A)
    nodes = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    op = ctx.rbf_operator_init(nodes, n, n, 1.0, 0.0, R.RBF_ASSEMBLED, R.RBF_FP64, R.RBF_FORM_C, Ad, lda)
    op._keep_fx = (Ad, nodes)
    return op


def test_fx_products_scaled_rows_and_columns(ctx, R):
    """Rows and columns scaled over 2^-40 .. 2^40, zero rows / columns, negative entries."""
    n = 1537
    rng = np.random.default_rng(5)
    A = rng.normal(size=(n, n))
    A *= np.ldexp(1.0, rng.integers(-40, 41, n))[:, None]
    A *= np.ldexp(1.0, rng.integers(-40, 41, n))[None, :]
    A[7, :] = 0.0
    A[:, 11] = 0.0
    A[rng.random((n, n)) < 0.01] = 0.0
    op = _write_matrix(ctx, R, A)
    f = rng.normal(size=n) * np.ldexp(1.0, rng.integers(-20, 21, n))
    check_first_step(ctx, R, A, op, f, "scaled", samples=48)


def test_fx_products_subnormal_and_huge(ctx, R):
    """Entries near both ends of the FP64 range in different rows (the largest
    ones small enough that GKB's sums of squares stay finite)."""
    n = 300
    rng = np.random.default_rng(6)
    A = rng.normal(size=(n, n))
    A[:50] *= 1e-300
    A[50:60] *= 1e-310  # subnormal entries
    A[60:70] *= 1e150
    op = _write_matrix(ctx, R, A)
    f = rng.normal(size=n)
    check_first_step(ctx, R, A, op, f, "range", samples=n)


def test_fx_nonfinite_entry_breaks_down(ctx, R):
    n = 200
    rng = np.random.default_rng(7)
    A = rng.normal(size=(n, n))
    A[17, 23] = np.inf
    op = _write_matrix(ctx, R, A)
    st, *_ = R.make_state(torch, n, 5)
    ctx.rbf_gkb(op, dev(rng.normal(size=n)), 5, st)
    assert st.breakdown == 3


@pytest.mark.parametrize("n,ni,steps", [(2049, 1500, 60), (8000, 5598, 40)])
def test_fx_gkb_matches_fma_products(ctx, R, n, ni, steps):
    """GKB with the fixed-point products against GKB with FP64 FMA products and
    the oracle: the scalars to rel 1e-10 up to l_stable (the first step where
    the oracle's own MGS2 and CGS2 runs differ by 1e-12)."""
    ns = random_nodes(n, ni, 17 * n)
    c, k = 0.2, 5.0
    op, _ = gpu_operator(ctx, R, ns, c, k)
    f = np.random.default_rng(n + 3).normal(size=n)
    st1, W1, Z1, a1, b1 = R.make_state(torch, n, steps)
    ctx.rbf_gkb(op, dev(f), steps, st1)
    cf = R.Context(0, fma_products=1)
    try:
        opf = cf.rbf_operator_init(op._keep_fx[1], n, ni, c, k, R.RBF_ASSEMBLED, R.RBF_FP64, R.RBF_FORM_C,
                                   op._keep_fx[0], op.lda)
        st2, W2, Z2, a2, b2 = R.make_state(torch, n, steps)
        cf.rbf_gkb(opf, dev(f), steps, st2)
        torch.cuda.synchronize()
    finally:
        cf.close()
    a1, b1, a2, b2 = (t.cpu().numpy() for t in (a1, b1, a2, b2))
    A = OM.assemble(ns.X, ni, c, k)  # the oracle's own matrix
    g1 = OG.gkb(A, None, f, steps, reorth="mgs2")
    g2 = OG.gkb(A, None, f, steps, reorth="cgs2")
    l = min(g1.steps_done, g2.steps_done, st1.steps_done, st2.steps_done)
    rel = np.maximum(np.abs(g1.alpha[:l] - g2.alpha[:l]) / g1.alpha[:l],
                     np.abs(g1.beta[1:l + 1] - g2.beta[1:l + 1]) / np.maximum(g1.beta[1:l + 1], 1e-300))
    bad = np.flatnonzero(rel > 1e-12)
    ls = max(1, int(bad[0]) if len(bad) else l)
    for al, be in ((a1, b1), (a2, b2)):
        assert np.max(np.abs(al[:ls] - g1.alpha[:ls]) / g1.alpha[:ls]) < 1e-10
        assert np.max(np.abs(be[:ls + 1] - g1.beta[:ls + 1]) / g1.beta[:ls + 1]) < 1e-10
    print(f"n = {n}: fixed point vs FMA products, alpha rel diff "
          f"{np.max(np.abs(a1[:ls] - a2[:ls]) / a2[:ls]):.1e} for j <= l_stable = {ls}")
    # the Golub-Kahan relations of the fixed-point run (Algorithm 1)
    W1, Z1 = W1.cpu().numpy().T, Z1.cpu().numpy().T
    ld = st1.steps_done
    C = np.zeros((ld + 1, ld))
    C[np.arange(ld), np.arange(ld)] = a1[:ld]
    C[np.arange(1, ld + 1), np.arange(ld)] = b1[1:ld + 1]
    nA = np.linalg.norm(A)
    assert np.linalg.norm(A @ Z1[:, :ld] - W1[:, :ld + 1] @ C) / nA < 1e-12
    assert np.linalg.norm(A.T @ W1[:, :ld] - Z1[:, :ld] @ C[:ld].T) / nA < 1e-12


def test_fx_workspace_cap_falls_back_to_fma(R):
    """A workspace cap without room for the fixed-point copies: same run, FMA products."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n, steps = 700, 20
    ns = random_nodes(n, 500, 3)
    c0 = R.Context(0)
    base = c0.rbf_workspace_bytes(n, steps, R.RBF_ASSEMBLED, R.RBF_FP64)
    c0.close()
    fx_bytes = 2 * n * R.padded_lda(n, R.RBF_FP64) * 8
    cap = base - fx_bytes + (1 << 20)
    outs = []
    for opts in ({"workspace_cap": cap}, {"fma_products": 1}):
        cx = R.Context(0, **opts)
        try:
            op, _ = gpu_operator(cx, R, ns, 0.4, 2.0)
            st, W, Z, al, be = R.make_state(torch, n, steps)
            cx.rbf_gkb(op, dev(np.ones(n)), steps, st)
            torch.cuda.synchronize()
            outs.append((al.cpu().numpy(), be.cpu().numpy()))
        finally:
            cx.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
