"""One regularized solve through the C ABI: assemble -> GKB -> HKT / Ine-TSVD
-> lift -> evaluate.  Argument marshalling and buffer allocation only (torch
tensors on the context's device); every arithmetic step runs in librbfkr.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import rbfkr as R


@dataclass
class Problem:
    """Device-resident inputs of one solve."""
    nodes: object          # torch float64 [3][n]
    n: int
    n_interior: int
    c: float
    k: float
    f: object              # torch float64 [n]
    points: object = None  # torch float64 [3][m]
    m: int = 0


@dataclass
class Buffers:
    A: object = None
    lda: int = 0
    state: object = None
    coef: object = None
    u: object = None
    curve: object = None
    keep: list = field(default_factory=list)


def to_device(torch, nodes_soa: np.ndarray, f: np.ndarray, points: np.ndarray | None, ni, c, k, device="cuda"):
    nd = torch.as_tensor(np.ascontiguousarray(nodes_soa), dtype=torch.float64, device=device)
    fd = torch.as_tensor(np.ascontiguousarray(f), dtype=torch.float64, device=device)
    pd, m = None, 0
    if points is not None:
        pd = torch.as_tensor(np.ascontiguousarray(points.T), dtype=torch.float64, device=device)
        m = points.shape[0]
    return Problem(nd, nodes_soa.shape[1], ni, c, k, fd, pd, m)


def allocate(torch, ctx: R.Context, prob: Problem, steps: int, precision: int, storage: int,
             device="cuda") -> Buffers:
    b = Buffers()
    if storage == R.RBF_ASSEMBLED:
        b.lda = R.padded_lda(prob.n, precision)
        dt = torch.float64 if precision == R.RBF_FP64 else torch.float32
        b.A = torch.empty((prob.n, b.lda), dtype=dt, device=device)
    b.state, *b.keep = R.make_state(torch, prob.n, steps, device)
    b.coef = torch.empty(prob.n, dtype=torch.float64, device=device)
    if prob.m:
        b.u = torch.empty(prob.m, dtype=torch.float64, device=device)
    # GCV / curvature on the context's lambda grid, or GCV_l(k) for k = 1..l
    b.curve = torch.empty(max(ctx.grid_j, steps), dtype=torch.float64, device=device)
    return b


def solve(ctx: R.Context, prob: Problem, buf: Buffers, steps: int, precision=R.RBF_FP64,
          storage=R.RBF_ASSEMBLED, method="hkt", rule=R.RBF_GCV, lam=0.0, rank=0,
          form=R.RBF_FORM_C, assemble=True):
    op = ctx.rbf_operator_init(prob.nodes, prob.n, prob.n_interior, prob.c, prob.k, storage, precision,
                               form, buf.A, buf.lda)
    if storage == R.RBF_ASSEMBLED and assemble:
        ctx.rbf_assemble(op)
    ctx.rbf_gkb(op, prob.f, steps, buf.state)
    if method == "hkt":
        info = ctx.rbf_hkt(buf.state, rule, lam, buf.coef, buf.curve)
    else:
        info = ctx.rbf_ine_tsvd(buf.state, rank, buf.coef, buf.curve)
    if prob.m:
        ctx.rbf_evaluate(op, buf.coef, prob.points, prob.m, buf.u)
    return op, info
