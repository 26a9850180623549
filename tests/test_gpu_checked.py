"""GPU: the bounds-checked build (librbfkr_checked.so, RBFKR_CHECKED=1).

Its device index tests must (a) report a failure through the normal error path
(a self-test index that fails by construction and touches no memory), and
(b) stay silent over runs of every kernel family at ragged sizes: assembly,
FP64 and mixed products (assembled and matrix-free), GKB with its half-step
kernels, concurrent lanes, the projected solves, the batched driver, the
reconstruction and the matrix-free tile pairs with folded partial slots.  The library is loaded once per process, so the checked runs
happen in a child process with RBFKR_CHECKED=1."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
import workloads as w
from paper_2511_09798_gb300 import rbfkr as R
lib = R.load()
assert lib.rbf_checked_build() == 1
ctx = R.Context(0)
ctx.rbf_check_selftest()
try:
    ctx.rbf_check()
    raise SystemExit("self-test index failure was not reported")
except R.RbfError as e:
    assert e.status == R.RBF_ERR_INTERNAL, e.status
    assert "ctx.cu" in str(e), str(e)
ctx.rbf_check()  # reported once, then clear
rng = np.random.Generator(np.random.PCG64(5))
sets = [w.cube_faces_random(n, 0.3, rng) for n in (37, 515, 1031, 2049)]
L = 24
for ns in sets:
    n = ns.n
    nodes = torch.as_tensor(ns.soa(), device="cuda")
    f = torch.as_tensor(w.plane_wave_rhs(ns, 2.0), device="cuda")
    P = torch.as_tensor(w.test_points(ns, 97).T.copy(), device="cuda")
    u = torch.empty(97, dtype=torch.float64, device="cuda")
    coef = torch.empty(n, dtype=torch.float64, device="cuda")
    for storage, prec in ((0, 0), (0, 1), (1, 1), (1, 0)):
        A, lda = None, 0
        if storage == 0:
            lda = R.padded_lda(n, prec)
            A = torch.full((n, lda), float("nan"), dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
        op = ctx.rbf_operator_init(nodes, n, ns.n_interior, 0.3, 2.0, storage, prec, 0, A, lda)
        if A is not None:
            ctx.rbf_assemble(op)
        st = R.make_state(torch, n, min(L, n))[0]
        ctx.rbf_gkb(op, f, min(L, n), st)
        ctx.rbf_hkt(st, R.RBF_GCV, 0.0, coef)
        ctx.rbf_ine_tsvd(st, 0, coef)
        ctx.rbf_evaluate(op, coef, P, 97, u)
ops, fs, sts, keep = [], [], [], []
for ns in sets[1:]:
    lda = R.padded_lda(ns.n, 0)
    A = torch.empty((ns.n, lda), dtype=torch.float64, device="cuda")
    nodes = torch.as_tensor(ns.soa(), device="cuda")
    ops.append(ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, 0.3, 2.0, 0, 0, 0, A, lda))
    keep.append((A, nodes))
    fs.append(torch.as_tensor(w.plane_wave_rhs(ns, 2.0), device="cuda"))
    sts.append(R.make_state(torch, ns.n, L)[0])
ctx.rbf_gkb_many(ops, fs, L, sts, assemble=True)
ctx.rbf_hkt_many(sts, R.RBF_GCV, 0.0, [torch.empty(s.n, dtype=torch.float64, device="cuda") for s in sets[1:]])
bt, kb = R.make_batch(torch, sets, [0.3] * 4, [2.0] * 4, [w.plane_wave_rhs(s, 2.0) for s in sets], L)
ctx.rbf_batch_gkb(bt, L)
T = int(kb["offsets"][-1])
ctx.rbf_batch_hkt(bt, R.RBF_GCV, torch.empty(T, dtype=torch.float64, device="cuda"))
# the matrix-free tile pairs with folded partial slots (26 000 nodes, FP32) and
# the 256-node blocks (9001 nodes), both products
for n, ni in ((26000, 20000), (9001, 6000)):
    X = np.random.default_rng(n).uniform(0, 1, (3, n))
    nodes = torch.as_tensor(X, device="cuda")
    op = ctx.rbf_operator_init(nodes, n, ni, 0.1, 8.0, 1, 1)
    x = torch.as_tensor(np.random.default_rng(1).normal(size=n), device="cuda")
    y = torch.empty_like(x)
    ctx.rbf_matvec(op, 0, x, y)
    ctx.rbf_matvec(op, 1, x, y)
ctx.rbf_check()
print("checked build: no index check failed")
'''


def test_checked_build_reports_and_stays_silent():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, RBFKR_CHECKED="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    print(r.stdout[-2000:], r.stderr[-4000:])
    assert r.returncode == 0
    assert "no index check failed" in r.stdout


def test_normal_build_compiles_the_checks_away():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09798_gb300 import rbfkr as R
    if os.environ.get("RBFKR_CHECKED") == "1":
        pytest.skip("this process loaded the checked build")
    assert R.load().rbf_checked_build() == 0
    ctx = R.Context(0)
    ctx.rbf_check_selftest()
    ctx.rbf_check()  # nothing to report
    ctx.close()
