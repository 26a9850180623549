"""Train the stop network on GKB runs the method itself generates, evaluate it
on held-out runs, and save the weights.

    python -m paper_2511_09798_gb300.train_stopnet --runs 10000 \\
        --n-lo 2000 --n-hi 16000 --gkb-steps 150 --out paper_2511_09798_gb300/stopnet_weights.npz

Training runs: node sets and (c, k) drawn like the batched sweep (cube or
sphere, N uneven in [n_lo, n_hi], c log-uniform in [0.05, 1], k uniform in
[1, 20]); the exact solution is a plane wave or the paper's Gaussian (half
each).  Every run is a batched mixed-precision GKB (one graph launch per
chunk), labelled from its error table (see ``learned``).  Evaluation: on
held-out runs, GCV-driven HKT and L-curve HKT at the full step count against
the learned stop, each timed end to end on the device and scored by the max
error against the exact solution at 500 test points.
"""
from __future__ import annotations

import argparse
import json
import os
import math
import sys
import time

import numpy as np


def generate(ctx, torch, insts, L, ells, m=500, chunk=96, t_stride=4):
    import workloads as w
    from . import learned
    feats, Es = [], []
    for s in range(0, len(insts), chunk):
        part = insts[s:s + chunk]
        cs = [p.params["c"] for p in part]
        ks = [p.params["k"] for p in part]
        fs = [w.instance_rhs(p) for p in part]
        pts = [w.test_points(p, m, seed=p.params["seed"] + 7) for p in part]
        ur = [w.instance_field(p, P) for p, P in zip(part, pts)]
        F, E, _ = learned.label_runs(ctx, torch, part, cs, ks, fs, pts, ur, L, ells, t_stride=t_stride)
        feats.append(F)
        Es.append(E)
    return np.concatenate(feats), np.concatenate(Es)


def evaluate(ctx, torch, net, insts, L, m=500):
    """Per held-out run: error and wall time of GCV-HKT(L), L-curve HKT(L) and
    the learned stop (mixed-precision matrix-free operator)."""
    import workloads as w
    from . import learned
    from . import rbfkr as R
    rows = []
    for ns in insts:
        c, k = ns.params["c"], ns.params["k"]
        f = torch.as_tensor(w.instance_rhs(ns), device="cuda")
        nodes = torch.as_tensor(ns.soa(), device="cuda")
        op = ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, c, k, R.RBF_MATRIX_FREE, R.RBF_MIXED)
        P = w.test_points(ns, m, seed=ns.params["seed"] + 7)
        ue = w.instance_field(ns, P)
        dP = torch.as_tensor(np.ascontiguousarray(P.T), device="cuda")
        u = torch.empty(m, dtype=torch.float64, device="cuda")
        coef = torch.empty(ns.n, dtype=torch.float64, device="cuda")

        def err():
            ctx.rbf_evaluate(op, coef, dP, m, u)
            return float(np.max(np.abs(u.cpu().numpy() - ue)) / np.max(np.abs(ue)))

        row = {"n": ns.n, "c": c, "k": k, "rhs": ns.params["rhs"], "domain": ns.domain}
        for name, rule in (("gcv", R.RBF_GCV), ("lcurve", R.RBF_LCURVE)):
            st, *_ = R.make_state(torch, ns.n, L)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.rbf_gkb(op, f, L, st)
            ctx.rbf_hkt(st, rule, 0.0, coef)
            torch.cuda.synchronize()
            row[f"{name}_s"] = time.perf_counter() - t0
            row[f"{name}_err"] = err()
            row[f"{name}_steps"] = st.steps_done
        st, *_ = R.make_state(torch, ns.n, L)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = learned.solve(ctx, op, f, net, st, coef)
        torch.cuda.synchronize()
        row["learned_s"] = time.perf_counter() - t0
        row["learned_err"] = err()
        row["learned_steps"] = info.steps
        row["learned_accepted"] = info.accepted
        row["learned_t"] = info.t_pred
        rows.append(row)
    return rows


def summarize(rows, by_domain=True):
    out = _summarize(rows)
    if by_domain:
        doms = sorted({r.get("domain", "?") for r in rows})
        if len(doms) > 1:
            out["by_domain"] = {d: _summarize([r for r in rows if r.get("domain", "?") == d]) for d in doms}
    return out


def _summarize(rows):
    g = np.array([[r["gcv_err"], r["lcurve_err"], r["learned_err"], r["gcv_s"], r["lcurve_s"], r["learned_s"],
                   r["learned_steps"], r["learned_accepted"]] for r in rows])
    eg, el, ex, tg, tl, tx, sx, acc = g.T
    return {
        "runs": len(rows),
        "accepted_frac": float(acc.mean()),
        "learned_steps_mean": float(sx.mean()),
        "time_ratio_vs_gcv_mean": float(np.mean(tx / tg)),
        "time_ratio_vs_lcurve_mean": float(np.mean(tx / tl)),
        "err_ratio_vs_gcv_median": float(np.median(ex / eg)),
        "err_ratio_vs_gcv_q90": float(np.quantile(ex / eg, 0.9)),
        "err_not_worse_than_gcv_frac": float(np.mean(ex <= 1.05 * eg)),
        "err_ratio_vs_lcurve_median": float(np.median(ex / el)),
        "err_ratio_vs_lcurve_q90": float(np.quantile(ex / el, 0.9)),
        "median_err": {"gcv": float(np.median(eg)), "lcurve": float(np.median(el)), "learned": float(np.median(ex))},
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--runs", type=int, default=10000)
    ap.add_argument("--eval-runs", type=int, default=100)
    ap.add_argument("--n-lo", type=int, default=2000)
    ap.add_argument("--n-hi", type=int, default=16000)
    ap.add_argument("--gkb-steps", type=int, default=150)
    ap.add_argument("--train-steps", type=int, default=8000)
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--rel-tol", type=float, default=0.25)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--pump-share", type=float, default=0.25,
                    help="share of casing-like node sets among the training and evaluation runs")
    ap.add_argument("--out", default=None)
    ap.add_argument("--summary", default=None)
    a = ap.parse_args(argv)
    import torch

    import workloads as w
    from . import learned
    from . import rbfkr as R

    ctx = R.Context(0)
    L = a.gkb_steps
    ells = list(range(10, L + 1, 10))
    tgrid = learned.grid_t(ctx.grid_j, ctx.grid_t_lo, ctx.grid_t_hi, 4)
    t0 = time.time()
    tr = w.stop_instances(a.runs, a.n_lo, a.n_hi, seed0=w.nodes.BASE_SEED + 600, pump_share=a.pump_share)
    F, E = generate(ctx, torch, tr, L, ells)
    torch.cuda.synchronize()
    t_gen = time.time() - t0
    Y = learned.make_labels(E, ells, tgrid, a.rel_tol)
    ok = np.all(np.isfinite(F), axis=1) & np.all(np.isfinite(Y), axis=1)
    t_min = float(np.min(Y[ok, 1])) - 0.5
    t_max = min(0.0, float(np.max(Y[ok, 1])) + 0.5)
    t1 = time.time()
    net, losses = learned.train(ctx, torch, F, Y, steps=a.train_steps, lr=a.lr, batch=a.batch, seed=a.seed,
                                log_every=max(1, a.train_steps // 10), l_min=10, l_max=L, window=5,
                                accept_tol=math.inf, t_min=t_min, t_max=t_max, fallback_rule=R.RBF_GCV,
                                z_max=6.0)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    ev = w.stop_instances(a.eval_runs, a.n_lo, a.n_hi, seed0=w.nodes.BASE_SEED + 50000, pump_share=a.pump_share)
    rows = evaluate(ctx, torch, net, ev, L)
    summ = {
        "training_runs": int(ok.sum()), "gkb_steps": L, "n_range": [a.n_lo, a.n_hi], "rel_tol": a.rel_tol,
        "pump_share": a.pump_share,
        "generate_s": t_gen, "train_s": t_train, "train_steps": a.train_steps, "losses": losses,
        "label_l_mean": float(np.exp(Y[ok, 0]).mean()), "t_range": [t_min, t_max],
        "eval": summarize(rows),
    }
    print(json.dumps(summ, indent=1))
    if a.out:
        net.save(a.out)
        # the same network in the layout the library reads from C (rbf_stopnet_load)
        learned.write_stopnet_file(a.out, os.path.splitext(a.out)[0] + ".bin")
    if a.summary:
        with open(a.summary, "w") as fh:
            json.dump({"summary": summ, "rows": rows}, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
