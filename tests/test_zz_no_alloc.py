"""The allocation-free transposed product against the context-based one.

``rbf_matvec_t_noalloc`` serves callers that cannot allocate device memory
(their device memory is reserved up front by another allocator, or they run a
latency-critical loop where cudaMalloc / cudaFree and the device-wide
synchronisation they may cause are not allowed).  It must give the same
A^T x as ``rbf_matvec`` with trans = 1, call after call, although its partial
sums live in one static device array shared by every call.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

import workloads as w
from oracle import mq as OM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09798_gb300 import rbfkr
    return rbfkr


def test_noalloc_matches_context_product_twice(R):
    ns = w.cube_faces_random(3001, 0.3, np.random.Generator(np.random.PCG64(17)))
    c, k = 0.2, 5.0
    n = ns.n
    ctx = R.Context(0)
    lda = R.padded_lda(n, R.RBF_FP64)
    A = torch.empty((n, lda), dtype=torch.float64, device="cuda")
    nodes = torch.as_tensor(ns.soa(), device="cuda")
    op = ctx.rbf_operator_init(nodes, n, ns.n_interior, c, k, R.RBF_ASSEMBLED, R.RBF_FP64, 0, A, lda)
    ctx.rbf_assemble(op)
    Ah = OM.assemble(ns.X, ns.n_interior, c, k)
    rng = np.random.default_rng(3)
    for call in range(2):  # two calls in a row share the static scratch
        x = rng.normal(size=n)
        xd = torch.as_tensor(x, device="cuda")
        y_ref = torch.empty(n, dtype=torch.float64, device="cuda")
        y = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        ctx.rbf_matvec(op, 1, xd, y_ref)
        R.rbf_matvec_t_noalloc(A, lda, n, xd, y)
        torch.cuda.synchronize()
        yr, yn = y_ref.cpu().numpy(), y.cpu().numpy()
        scale = np.abs(Ah).T @ np.abs(x)
        assert np.max(np.abs(yn - yr) / scale) < 1e-14, call
        assert np.max(np.abs(yn - Ah.T @ x) / scale) < 1e-14, call
    ctx.close()


def test_noalloc_rejects_sizes_beyond_the_scratch(R):
    A = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    # n = 70 000 needs at least 18 row chunks of n doubles > 2^20: rejected before any launch
    with pytest.raises(R.RbfError) as e:
        R.rbf_matvec_t_noalloc(A, 70000, 70000, x, x)
    assert e.value.status == R.RBF_ERR_INVALID
    with pytest.raises(R.RbfError):
        R.rbf_matvec_t_noalloc(A, 3, 4, x, x)  # lda < n
