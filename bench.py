#!/usr/bin/env python
"""Benchmark: GKB steps/s and time-to-HKT-solution on one GB300 (or N replicas).

Workload (default ``cube8000``): the N = 8000 Halton cube (21 x 21 face grid,
2402 Dirichlet nodes, 5598 scrambled-Halton interior nodes), plane wave
u = sin(k (x + y + z) / sqrt 3), FP64, assembled A (512 MB), 100 GKB steps, HKT
with GCV, u at 2000 seeded test points.  One bench step = the six solves
c in {0.1, 0.2, 0.5} x k in {2, 5}; each solve assembles A, runs GKB, the
projected SVD, GCV, the projected solve, the lift and the reconstruction.  The
six solves are independent: they run concurrently on `--lanes` streams of the
library context (rbf_gkb_many, rbf_hkt_many).

value = GKB steps completed / device time (all ranks, max time over ranks).
e2e   = the same metric through the C ABI with the step's inputs copied from
        pinned host memory and u copied back inside the timed region.
roofline: the dominant kernel is the matrix-vector product of the GKB; its
        launches are timed live with CUDA events on the launching streams, and
        the per-launch time is the union of the launch intervals divided by the
        launches (concurrent products overlap).  The FP64 product is bound by
        the FP64 pipe (1 FMA per 8-byte entry), so the bound is "alu" with the
        measured FP64 FMA peak 1.2573 TFLOP/s (2 FMA/clk/SM at 2.07 GHz); the
        HBM fraction is reported beside it.
re_exact: Re = max |u - u_exact| / max |u_exact| of every solve at the test
        points; gaussian_variant: the same solve for the cube example's
        Gaussian exact solution (a field HKT resolves), timed one solve after
        another; forms_comparison: 24 uneven instances with Gaussian exact
        solutions solved by every form (FP64, mixed, batched, learned stop):
        time to solution and error against the exact solution.

``--impl reference`` times the FP64 CPU oracle (test infrastructure) on the
host cores, one full solve of the same workload per step.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GKB steps/s and time-to-HKT-solution at N (fraction of HBM/FP32 roofline)"
# FP64 FMA pipe of the GB300, measured by `bench.py --workload fp64-pipe-probe`
# (1.998 FMA/clk/SM at 2070 MHz; nominal 152 x 2 FMA/clk x 2 flop x 2.07 GHz = 1.2586)
FP64_PEAK_TFLOPS = 1.2573
FP64_PEAK_SOURCE = ("measured: FP64 FMA probe, 1.2573 TFLOP/s = 1.998 FMA/clk/SM at 2070 MHz "
                    "(bench.py --workload fp64-pipe-probe)")
FP32_LANE_TOPS = 152 * 128 * 2.07e9 / 1e12  # FP32 pipe: one operation per lane per clock


# DRAM bytes (read + write) per launch of the dominant product kernel, from one
# ncu capture of that kernel at the workload's size (dram__bytes_read.sum +
# dram__bytes_write.sum); None where the kernel changed after its capture.
FX_MAX_N = 16384  # FP64 assembled operators up to this size take the fixed-point products
MEASURED_TRAFFIC = {
    ("cube8000", 0): 512.113e6 + 0.166e6,                      # k_gemv_flat_f64
    ("cube8000", 1): 512.116e6 + 4.010e6,                      # k_gemv_t_f64
    ("cube8000-fx", 0): 512.184e6 + 3.377e6,                   # k_gemv_flat_fx
    ("cube8000-fx", 1): 512.147e6 + 3.250e6,                   # k_gemv_t_fx
    ("sphere20000-mixed-assembled", 0): 1600.665e6 + 4.324e6,  # k_gemv_nseg_f32
    ("sphere20000-mixed-assembled", 1): 1600.146e6 + 3.266e6,  # k_gemv_t_f32
}


def mf_pair_ops(n, n_interior):
    """FP32 pipe operations of one single-instance matrix-free product, which
    evaluates each unordered node pair once (s = |X_i - X_j|^2 + c^2 and its
    rsqrt are shared by A_ij and A_ji): 3 differences and 3 FMA for s, the
    entry factors the two row types need (PDE: rs^2, two FMA, one multiply;
    Dirichlet: rs s; a mixed pair both) and two accumulate FMA; the diagonal
    entries one accumulate each.  The rsqrt goes to the MUFU unit."""
    ni, nb = n_interior, n - n_interior
    return (12 * ni * (ni - 1) / 2 + 9 * nb * (nb - 1) / 2 + 13 * ni * nb + 11 * ni + 8 * nb)


def mf_pair_ops_f64(n, n_interior):
    """FP64 pipe operations of one FP64 matrix-free product by tile pairs:
    per unordered node pair 3 differences, 3 FMA for s, 5 for the refined
    s^{-1/2} (its FP32 estimate and the conversions around it not counted),
    the entry factors (PDE: rs^2, two FMA, one multiply; Dirichlet: rs s; a
    mixed pair both) and two accumulate FMA; the diagonal one accumulate."""
    ni, nb = n_interior, n - n_interior
    return (17 * ni * (ni - 1) / 2 + 14 * nb * (nb - 1) / 2 + 18 * ni * nb + 16 * ni + 13 * nb)


def mf_roofline(n, n_interior, avg_ms):
    """Roofline of the FP32 matrix-free product (tile pairs, mf_pair_ops)."""
    ent = n * n / (avg_ms / 1e3)
    ops = mf_pair_ops(n, n_interior) / (n * n)
    tops = ent * ops / 1e12
    return {"bound": "alu", "achieved": round(tops, 3), "peak": round(FP32_LANE_TOPS, 3),
            "unit": "T FP32-pipe ops/s", "frac": round(tops / FP32_LANE_TOPS, 4), "traffic": None,
            "entries_per_s": ent, "ops_per_entry": round(ops, 3),
            "peak_source": "152 SMs x 128 FP32 lanes x 2.07 GHz (unit counts and max clock)"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "_fallback": True}


def reduce_over_ranks(ms, work, device="cpu"):
    """Whole-job figures of a replicated run: the slowest rank's time and the
    work summed over ranks (one process per GPU; a no-op without a process
    group).  The all-reduces run on `device` (CUDA tensors for NCCL, CPU
    tensors for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), work
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    d = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(d, op=dist.ReduceOp.SUM)
    return float(t.item()), (int(d.item()) if isinstance(work, int) else float(d.item()))


def rank_barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


# --------------------------------------------------------------------------- workloads
def workload(name):
    import numpy as np

    import workloads as w
    if name == "cube1000":
        ns = w.preset("cube1000")
        cases = [(0.3, 2.0)]
        steps, prec, storage = 40, "fp64", "assembled"
    elif name == "cube8000":
        ns = w.preset("cube8000")
        cases = [(c, k) for c in (0.1, 0.2, 0.5) for k in (2.0, 5.0)]
        steps, prec, storage = 100, "fp64", "assembled"
    elif name == "cube8000-fp64-mf":
        ns = w.preset("cube8000")
        cases = [(0.2, 5.0)]
        steps, prec, storage = 100, "fp64", "matrix_free"
    elif name == "cube8000-mixed-mf":
        ns = w.preset("cube8000")
        cases = [(c, k) for c in (0.1, 0.2, 0.5) for k in (2.0, 5.0)]
        steps, prec, storage = 100, "mixed", "matrix_free"
    elif name == "sphere20000":
        ns = w.preset("sphere20000")
        cases = [(0.15, 10.0)]
        steps, prec, storage = 150, "mixed", "matrix_free"
    elif name == "sphere20000-mixed-assembled":
        ns = w.preset("sphere20000")
        cases = [(0.15, 10.0)]
        steps, prec, storage = 150, "mixed", "assembled"
    else:
        raise SystemExit(f"unknown workload {name}")
    P = w.test_points(ns)
    fs = {k: w.plane_wave_rhs(ns, k) for k in sorted({k for _, k in cases})}
    exact = {k: w.plane_wave(P, k) for k in fs}
    return dict(name=name, ns=ns, cases=cases, steps=steps, precision=prec, storage=storage,
                points=P, fs=fs, exact=exact, exact_name="plane wave sin(k (x + y + z) / sqrt 3)", np=np)


def gaussian_variant(R, ctx, wl, nodes_d, pts_d, stream, dev, reps=5):
    """The same N = 8000 FP64 assembled solve (assemble, GKB, HKT with GCV, u)
    for the Gaussian exact solution exp(-|X|^2 / 20) of the cube example
    (Sec. 5, Example 1) at k = 3, with c = 2: a field that HKT resolves (the
    plane waves of the headline are not resolved by 100 GKB steps).  Device
    time per solution over `reps` solves, and Re at the test points."""
    import numpy as np
    import torch

    import workloads as w
    ns, L = wl["ns"], wl["steps"]
    n, m = ns.n, wl["points"].shape[0]
    c, k, sigma = 2.0, 3.0, 20.0
    f = torch.as_tensor(w.gaussian_rhs(ns, sigma, k), device=dev)
    ue = w.gaussian(wl["points"], sigma)
    lda = R.padded_lda(n, R.RBF_FP64)
    A = torch.empty((n, lda), dtype=torch.float64, device=dev)
    op = ctx.rbf_operator_init(nodes_d, n, ns.n_interior, c, k, R.RBF_ASSEMBLED, R.RBF_FP64, R.RBF_FORM_C, A, lda)
    st = R.make_state(torch, n, L, dev)[0]
    coef = torch.empty(n, dtype=torch.float64, device=dev)
    u = torch.empty(m, dtype=torch.float64, device=dev)

    def solve():
        ctx.rbf_assemble(op)
        ctx.rbf_gkb(op, f, L, st)
        inf = ctx.rbf_hkt(st, R.RBF_GCV, 0.0, coef)
        ctx.rbf_evaluate(op, coef, pts_d, m, u)
        return inf

    solve()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        info = solve()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    re = float(np.max(np.abs(u.cpu().numpy() - ue)) / np.max(np.abs(ue)))
    return {"exact": "Gaussian exp(-|X|^2 / 20)", "c": c, "k": k, "gkb_steps": st.steps_done, "rule": "gcv",
            "solves_timed": reps, "time_to_solution_ms": round(ms / reps, 3),
            "gkb_steps_per_s": round(st.steps_done * reps / (ms / 1e3), 1), "re_exact": round(re, 8),
            "lambda_over_s1_log10": round(float(np.log10(info.lambda_ / info.sigma1)), 3),
            "timing": "one solve after another through rbf_assemble / rbf_gkb / rbf_hkt / rbf_evaluate, "
                      "CUDA events around the solves"}


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2511_09798_gb300 import rbfkr as R

    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    wl = workload(args.workload)
    ns, cases, L = wl["ns"], wl["cases"], wl["steps"]
    prec = R.RBF_FP64 if wl["precision"] == "fp64" else R.RBF_MIXED
    storage = R.RBF_ASSEMBLED if wl["storage"] == "assembled" else R.RBF_MATRIX_FREE
    stream = torch.cuda.current_stream()
    fma = int(bool(getattr(args, "fma_products", False)))
    ctx = R.Context(local_rank, stream=stream, timing=2, fma_products=fma)
    n, m = ns.n, wl["points"].shape[0]
    # device-resident inputs
    nodes_h = torch.from_numpy(ns.soa()).pin_memory()
    pts_h = torch.from_numpy(np.ascontiguousarray(wl["points"].T)).pin_memory()
    f_h = {k: torch.from_numpy(v).pin_memory() for k, v in wl["fs"].items()}
    nodes_d = nodes_h.to(dev)
    pts_d = pts_h.to(dev)
    f_d = {k: v.to(dev) for k, v in f_h.items()}
    lda = R.padded_lda(n, prec)
    adt = torch.float64 if prec == R.RBF_FP64 else torch.float32
    # one operator (and, assembled, one matrix) per (c, k) case: the cases are
    # independent solves, run concurrently on the context's lanes
    mats = [torch.empty((n, lda), dtype=adt, device=dev) if storage == R.RBF_ASSEMBLED else None for _ in cases]
    ops = [ctx.rbf_operator_init(nodes_d, n, ns.n_interior, c, k, storage, prec, R.RBF_FORM_C, Ac,
                                 lda if Ac is not None else 0) for (c, k), Ac in zip(cases, mats)]
    states = [R.make_state(torch, n, L, dev)[0] for _ in cases]
    coef_all = torch.empty((len(cases), n), dtype=torch.float64, device=dev)
    coefs = list(coef_all)
    # consecutive cases with the same c share Phi(P, X) (it does not depend on
    # k): their reconstructions are one rbf_evaluate_many call
    ev_groups = []
    for ci, (c_, _) in enumerate(cases):
        if ev_groups and cases[ev_groups[-1][0]][0] == c_:
            ev_groups[-1][1] += 1
        else:
            ev_groups.append([ci, 1])
    fs_case = [f_d[k] for _, k in cases]
    A = mats[0]
    st = states[0]
    coef = coefs[0]
    u_d = torch.empty((len(cases), m), dtype=torch.float64, device=dev)
    u_h = torch.empty((len(cases), m), dtype=torch.float64).pin_memory()
    last_infos = []

    def one_step(e2e=False):
        if e2e:
            nodes_d.copy_(nodes_h, non_blocking=True)
            pts_d.copy_(pts_h, non_blocking=True)
            for k in f_d:
                f_d[k].copy_(f_h[k], non_blocking=True)
        # assemble + GKB (Algorithm 1) of every case, then the projected solves
        # (Algorithm 4, GCV) and the reconstructions
        ctx.rbf_gkb_many(ops, fs_case, L, states, lanes=args.lanes, assemble=storage == R.RBF_ASSEMBLED)
        last_infos[:] = ctx.rbf_hkt_many(states, R.RBF_GCV, 0.0, coefs, lanes=args.lanes)
        for c0, cnt in ev_groups:
            ctx.rbf_evaluate_many(ops[c0], coef_all[c0], n, cnt, pts_d, m, u_d[c0])
        if e2e:
            u_h.copy_(u_d, non_blocking=True)
        return sum(s_.steps_done for s_ in states)

    def timed(k_steps, e2e):
        rank_barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        done = 0
        for _ in range(k_steps):
            done += one_step(e2e)
        e1.record(stream)
        torch.cuda.synchronize()
        return reduce_over_ranks(e0.elapsed_time(e1), done, dev)

    for _ in range(args.warmup):
        one_step()
    ctx.rbf_get_counters(reset=True)
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
    ms, done = timed(args.steps, False)
    clocks = sampler.stop() if sampler else None
    cnt = ctx.rbf_get_counters(reset=True)
    # accuracy of the timed solves against the exact solution (eq. rel_error)
    uh = u_d.cpu().numpy()
    re_exact = [float(np.max(np.abs(uh[ci] - wl["exact"][k])) / np.max(np.abs(wl["exact"][k])))
                for ci, (_, k) in enumerate(cases)]
    t_chosen = [float(np.log10(x.lambda_ / x.sigma1)) for x in last_infos]
    ms_e2e, done_e2e = timed(args.steps, True)
    gauss = gaussian_variant(R, ctx, wl, nodes_d, pts_d, stream, dev) if wl["name"] == "cube8000" else None
    ctx.rbf_get_counters(reset=True)
    # the forms of the method on uneven instances whose field HKT resolves:
    # time to solution and error against the exact solution (after the timed region)
    forms = forms_comparison(local_rank) if wl["name"] == "cube8000" and not args.no_forms else None
    mf_roof = mf_product_roofline(local_rank) if wl["name"] == "cube8000" and not args.no_forms else None
    # phase shares (separate context with synchronising per-phase timers)
    ctx_ph = R.Context(local_rank, stream=stream, timing=1, fma_products=fma)
    phases = {}
    for ci, (c, k) in enumerate(cases[:1]):
        op = ctx_ph.rbf_operator_init(nodes_d, n, ns.n_interior, c, k, storage, prec, R.RBF_FORM_C,
                                      A, lda if A is not None else 0)
        t0 = time.perf_counter()
        if A is not None:
            ctx_ph.rbf_assemble(op)
        ctx_ph.rbf_gkb(op, f_d[k], L, st)
        ctx_ph.rbf_hkt(st, R.RBF_GCV, 0.0, coef)
        ctx_ph.rbf_evaluate(op, coef, pts_d, m, u_d[ci])
        phases = ctx_ph.rbf_get_timings()
    ctx_ph.close()
    methods = all_methods(ctx, wl, nodes_d, pts_d, f_d, A, lda, storage, prec, st, coef, stream) \
        if wl["name"] == "cube1000" else None
    if rank != 0:
        return None
    peaks = measured_peaks()
    solves = args.steps * len(cases) * world
    value = done / (ms / 1e3)
    # dominant kernel: the GKB products (A z and A^T w, the same algorithmic work
    # per launch).  Products of concurrent runs overlap, so the per-launch time
    # is the union of all product launch intervals (CUDA events on the lanes'
    # streams) divided by the launches: the device time the products occupied.
    p_ms, p_cnt = cnt["product_ms"], cnt["product_launches"]
    kinds = ["gemv_n (p = A z)", "gemv_t (r = A^T w)"]
    dom = 0 if p_ms[0] >= p_ms[1] else 1
    n_prod = max(1, p_cnt[0] + p_cnt[1])
    both_avg_ms = (p_ms[0] + p_ms[1]) / n_prod
    avg_ms = cnt["product_busy_ms"] / n_prod
    s = 8 if prec == R.RBF_FP64 else 4
    if storage == R.RBF_ASSEMBLED:
        alg_bytes = s * n * n
        gbs = alg_bytes / (avg_ms / 1e3) / 1e9
        fixed_point = prec == R.RBF_FP64 and not fma and n <= FX_MAX_N
        if fixed_point:
            # exact integer fixed-point products (k_gemv_flat_fx, k_gemv_t_fx): the
            # FP64 pipe is out of the inner loop and HBM is the bound
            tflops = 2.0 * n * n / (avg_ms / 1e3) / 1e12
            roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                    "frac": round(gbs / peaks.get("hbm_gbs", 6790.7), 4), "traffic": None,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                    "arithmetic": "int64 fixed point: 6 IMAD.WIDE (32x32+64) per 8-byte entry, exact sums, "
                                  "one FP64 rounding per partial",
                    "fp64_fma_equivalent_tflops": round(tflops, 4),
                    "fp64_fma_equivalent_frac_of_fp64_peak": round(tflops / FP64_PEAK_TFLOPS, 4)}
        elif prec == R.RBF_FP64:
            tflops = 2.0 * n * n / (avg_ms / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": round(tflops, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                    "unit": "TFLOP/s", "frac": round(tflops / FP64_PEAK_TFLOPS, 4), "traffic": None,
                    "pipe": "fp64 (2 FMA/clk/SM; 1 FMA per 8-byte entry)",
                    "peak_source": FP64_PEAK_SOURCE,
                    "hbm_achieved_gbs": round(gbs, 1), "hbm_peak_gbs": peaks.get("hbm_gbs"),
                    "hbm_frac": round(gbs / peaks.get("hbm_gbs", 6790.7), 4)}
        else:
            roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                    "frac": round(gbs / peaks.get("hbm_gbs", 6790.7), 4), "traffic": None,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
    elif prec == R.RBF_FP64:  # FP64 regeneration by tile pairs (mf_pair_ops_f64)
        ent = n * n / (avg_ms / 1e3)
        peak = 152 * 2 * 2.07e9 / 1e12
        ops = mf_pair_ops_f64(n, ns.n_interior)
        tops = ops / (avg_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": round(tops, 4), "peak": round(peak, 4), "unit": "T FP64-pipe ops/s",
                "frac": round(tops / peak, 4), "traffic": None, "entries_per_s": ent,
                "ops_per_entry": round(ops / (n * n), 3),
                "peak_source": "152 SMs x 2 FP64 ops/clk x 2.07 GHz (unit counts and max clock)"}
    else:
        roof = mf_roofline(n, ns.n_interior, avg_ms)
    fixed_point = storage == R.RBF_ASSEMBLED and prec == R.RBF_FP64 and not fma and n <= FX_MAX_N
    roof["traffic"] = MEASURED_TRAFFIC.get((wl["name"] + ("-fx" if fixed_point else ""), dom))
    kname = ("k_gemv_flat_fx (p = A z) and k_gemv_t_fx (r = A^T w), int64 fixed point" if fixed_point
             else "gemv_n (p = A z) and gemv_t (r = A^T w)" if storage == R.RBF_ASSEMBLED
             else ("k_mf_sym_f64" if prec == R.RBF_FP64 else "k_mf_sym") + " (p = A z, r = A^T w, matrix-free)")
    roof.update({"kernel": kname, "avg_launch_ms": round(avg_ms, 5),
                 "avg_launch_ms_how": "union of the product launch intervals / launches (CUDA events on the "
                                      "launching streams, timed region)",
                 "avg_launch_ms_events": round(both_avg_ms, 5), "launches_timed": int(p_cnt[0] + p_cnt[1]),
                 "algorithmic_per_launch": (f"{s * n * n} bytes, {2 * n * n} flop" if storage == R.RBF_ASSEMBLED
                                            else f"{n * n} entries")})
    h2d = nodes_h.numel() * 8 + pts_h.numel() * 8 + sum(v.numel() * 8 for v in f_h.values())
    d2h = u_h.numel() * 8
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GKB steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == R.RBF_FP64 else "f32+f64",
        "data": "synthetic",
        "config": {"workload": wl["name"], "n": n, "n_interior": ns.n_interior, "gkb_steps": L,
                   "cases_c_k": cases, "solves_per_step": len(cases), "precision": wl["precision"],
                   "storage": wl["storage"], "rule": "gcv", "test_points": m,
                   "products": ("int64 fixed point (exact sums, FP64 in and out)" if fixed_point
                                else "FP64 FMA" if prec == R.RBF_FP64 and storage == R.RBF_ASSEMBLED
                                else "matrix-free" if storage == R.RBF_MATRIX_FREE else "FP32"),
                   "parallelism": f"replicas x{world}; the step's independent solves on "
                                  f"{args.lanes or min(len(cases), 8)} streams",
                   "l2": "inputs larger than L2 (A or node set streamed each product)"},
        # amortized: the step's device time over its solves (solves run concurrently)
        "time_to_solution_ms": round(ms / (args.steps * len(cases)), 3),
        "lanes": args.lanes or min(len(cases), 8),
        "re_exact": {"per_case": [round(x, 6) for x in re_exact], "max": round(max(re_exact), 6),
                     "exact": wl["exact_name"], "test_points": m},
        "lambda_over_s1_log10": [round(x, 3) for x in t_chosen],
        "gaussian_variant": gauss,
        "forms_comparison": forms,
        "matrix_free_roofline": mf_roof,
        "gkb_steps_done": done, "solves": solves,
        "roofline": roof,
        "e2e": {"value": round(done_e2e / (ms_e2e / 1e3), 2), "unit": "GKB steps/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": round(ms_e2e / args.steps, 3)},
        "gpu_launches": int(cnt["launches"]),
        "phase_ms_one_solve": {k: round(v, 3) for k, v in phases.items() if k.endswith("_ms")},
        "methods": methods,
        "clocks": clocks,
    }
    ctx.close()
    return out


def all_methods(ctx, wl, nodes_d, pts_d, f_d, A, lda, storage, prec, st, coef, stream):
    """Every method of the paper on the first (c, k) case, each timed once on the
    device (after the timed region) with its max error against the exact plane
    wave: full-SVD Tikhonov and TSVD (Algorithm 3, GCV), Ine-TSVD and HKT on
    l GKB steps (Algorithms 2 and 4, GCV and L-curve), LSQR early stopping."""
    import numpy as np
    import torch

    import workloads as w
    from paper_2511_09798_gb300 import rbfkr as R
    ns, (c, k), L = wl["ns"], wl["cases"][0], wl["steps"]
    n, m = ns.n, wl["points"].shape[0]
    ue = w.plane_wave(wl["points"], k)
    u = torch.empty(m, dtype=torch.float64, device=nodes_d.device)
    op = ctx.rbf_operator_init(nodes_d, n, ns.n_interior, c, k, storage, prec, R.RBF_FORM_C, A,
                               lda if A is not None else 0)
    if A is not None:
        ctx.rbf_assemble(op)
    out = {}

    def timed(name, fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = fn()
        ctx.rbf_evaluate(op, coef, pts_d, m, u)
        e1.record(stream)
        torch.cuda.synchronize()
        err = float(np.max(np.abs(u.cpu().numpy() - ue)) / np.max(np.abs(ue)))
        out[name] = {"ms": round(e0.elapsed_time(e1), 3), "max_err_vs_exact": err}
        if info is not None:
            out[name].update({"lambda": info.lambda_, "rank": info.rank, "steps": info.steps})

    f = f_d[k]
    timed("tikhonov_full_gcv", lambda: ctx.rbf_tikhonov(op, f, R.RBF_GCV, 0.0, coef))
    timed("tsvd_full_gcv", lambda: ctx.rbf_tsvd(op, f, 0, coef))

    def gkb_then(solve):
        ctx.rbf_gkb(op, f, L, st)
        return solve()
    timed("hkt_gcv", lambda: gkb_then(lambda: ctx.rbf_hkt(st, R.RBF_GCV, 0.0, coef)))
    timed("hkt_lcurve", lambda: gkb_then(lambda: ctx.rbf_hkt(st, R.RBF_LCURVE, 0.0, coef)))
    timed("ine_tsvd_gcv", lambda: gkb_then(lambda: ctx.rbf_ine_tsvd(st, 0, coef)))
    timed("lsqr_lcurve", lambda: gkb_then(lambda: ctx.rbf_lsqr(st, R.RBF_LCURVE, 0, coef)))
    timed("lsqr_gcv", lambda: gkb_then(lambda: ctx.rbf_lsqr(st, R.RBF_GCV, 0, coef)))
    return out


# --------------------------------------------------------------------------- batch (96 instances)
def run_batch(args, rank, world, local_rank):
    """96 uneven instances (cube/sphere, N in [2000, 16000], c log-uniform in
    [0.05, 1], k in [1, 20], plane-wave direction on S^2), mixed precision,
    matrix-free FP32 products, 150 GKB steps, HKT with GCV, u at 200 points per
    instance; one bench step = the whole batch through the C ABI."""
    import numpy as np
    import torch

    import workloads as w
    from paper_2511_09798_gb300 import rbfkr as R

    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    inst = w.batch_instances(96)
    L = 150
    fs = [w.plane_wave_rhs(s, s.params["k"], s.params["d"]) for s in inst]
    ctx = R.Context(local_rank, stream=torch.cuda.current_stream())
    bt, keep = R.make_batch(torch, inst, [s.params["c"] for s in inst], [s.params["k"] for s in inst], fs, L, dev)
    T = int(keep["offsets"][-1])
    coef = torch.empty(T, dtype=torch.float64, device=dev)
    m = 200
    pts = [w.test_points(s, m, seed=s.params["seed"] + 7) for s in inst]
    P = torch.as_tensor(np.concatenate([p.T.ravel() for p in pts]), device=dev)
    u = torch.empty(m * len(inst), dtype=torch.float64, device=dev)

    learned_arm = args.workload == "batch96-learned"
    snet = None
    if learned_arm:
        from paper_2511_09798_gb300 import learned
        net = learned.StopNet.load(torch, os.path.join(ROOT, "paper_2511_09798_gb300", "stopnet_weights.npz"),
                                   device=dev)
        snet = net.c_struct()

    def one(use_learned=learned_arm):
        if use_learned:
            infos = ctx.rbf_batch_learned_hkt(bt, snet, coef)
            lam = [x.solve.lambda_ for x in infos]
        else:
            ctx.rbf_batch_gkb(bt, L)
            lam = ctx.rbf_batch_hkt(bt, R.RBF_GCV, coef)
        ctx.rbf_batch_evaluate(bt, coef, P, [m] * len(inst), u)
        return sum(bt.steps_done[b] for b in range(len(inst))), lam

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    ctx.rbf_get_counters(reset=True)
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
    rank_barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    steps_total = 0
    entries = 0  # matrix entries regenerated by the products (the learned arm's first 10 steps included)
    for _ in range(args.steps):
        st, lam = one()
        steps_total += st
        entries += sum(2 * (bt.steps_done[b] + (10 if learned_arm else 0)) * inst[b].n ** 2
                       for b in range(len(inst)))
    e1.record()
    torch.cuda.synchronize()
    ms, instances_all = reduce_over_ranks(e0.elapsed_time(e1), len(inst) * args.steps, dev)
    clocks = sampler.stop() if sampler else None
    cnt = ctx.rbf_get_counters(reset=True)

    def errors():
        uh = u.cpu().numpy().reshape(len(inst), m)
        out = []
        for b, s_ in enumerate(inst):
            ue = w.plane_wave(pts[b], s_.params["k"], s_.params["d"])
            out.append(float(np.max(np.abs(uh[b] - ue)) / np.max(np.abs(ue))))
        return out

    errs = errors()
    mean_steps = steps_total / (len(inst) * args.steps)
    tune = ctx.rbf_get_tuning()

    # end to end: every step copies its inputs (nodes, f, test points) from
    # pinned host memory and reads u back
    nodes_h, f_h, P_h = (t.cpu().pin_memory() for t in (keep["nodes"], keep["f"], P))
    u_h = torch.empty(u.shape, dtype=u.dtype).pin_memory()
    rank_barrier()
    torch.cuda.synchronize()
    x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x0.record()
    for _ in range(args.steps):
        keep["nodes"].copy_(nodes_h, non_blocking=True)
        keep["f"].copy_(f_h, non_blocking=True)
        P.copy_(P_h, non_blocking=True)
        one()
        u_h.copy_(u, non_blocking=True)
    x1.record()
    torch.cuda.synchronize()
    ms_e2e, inst_e2e = reduce_over_ranks(x0.elapsed_time(x1), len(inst) * args.steps, dev)
    h2d = (nodes_h.numel() + f_h.numel() + P_h.numel()) * 8
    d2h = u_h.numel() * 8

    # dominant kernel: the batched matrix-free products, timed live by the
    # autotuner (one A and one A^T product over the whole batch, best config)
    roof = None
    if tune.get("best_ms", 0) > 0:
        ops = int(sum(2 * mf_pair_ops(s_.n, s_.n_interior) for s_ in inst))
        tops = ops / (tune["best_ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": round(tops, 3), "peak": round(FP32_LANE_TOPS, 3),
                "unit": "T FP32-pipe ops/s", "frac": round(tops / FP32_LANE_TOPS, 4), "traffic": None,
                "kernel": "k_mf_batch (one A and one A^T product of all instances)",
                "avg_launch_ms": round(tune["best_ms"] / 2, 5),
                "timing": "the autotuner's CUDA-event timing of the chosen configuration, this run",
                "algorithmic_per_launch": f"{sum(s_.n * s_.n for s_ in inst)} entries, "
                                          f"{ops // 2} FP32-pipe ops (mf_pair_ops: each node pair once for "
                                          f"A_ij and A_ji)",
                "peak_source": "152 SMs x 128 FP32 lanes x 2.07 GHz (unit counts and max clock)"}
    # per-kernel times of one batch, launched directly with CUDA events around
    # every launch (a context with launch timing does not replay the graph):
    # the half-step kernel's roofline, and how much of the graph-replayed batch
    # is not kernel time (what a single persistent kernel could at most save)
    kern = None
    if not learned_arm:
        torch.cuda.synchronize()  # the GKB alone as the graph replays it
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record()
        ctx.rbf_batch_gkb(bt, L)
        q1.record()
        torch.cuda.synchronize()
        ms_graph_gkb = q0.elapsed_time(q1)
        ctx_t = R.Context(local_rank, stream=torch.cuda.current_stream(), timing=2)
        ctx_t.rbf_batch_gkb(bt, L)  # tunes on this context (untimed)
        ctx_t.rbf_get_counters(reset=True)
        torch.cuda.synchronize()
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record()
        ctx_t.rbf_batch_gkb(bt, L)
        k1.record()
        torch.cuda.synchronize()
        ct = ctx_t.rbf_get_counters(reset=True)
        ctx_t.close()
        ms_direct = k0.elapsed_time(k1)
        nh = max(1, ct["reorth_launches"])
        half_ms = ct["reorth_ms"] / nh
        prod_ms = sum(ct["product_ms"])
        done_b = [bt.steps_done[b] for b in range(len(inst))]
        # algorithmic work of one batched half-step, averaged over the run:
        # classical Gram-Schmidt applied twice against each active instance's
        # basis of M vectors is 2 passes x (dots + update) = 4 n_b M FP64 FMAs;
        # over a run M = j - 1 (r-side) and j (p-side), so the FMAs sum to
        # 4 n_b l_b^2.  Bytes: one read of every active basis (8 n_b l_b^2 over
        # the run) plus the vectors each half-step reads and writes (~5 x 8 n_b).
        fma = sum(4 * s_.n * l_b * l_b for s_, l_b in zip(inst, done_b)) / (2 * L)
        basis = sum(8 * s_.n * l_b * l_b for s_, l_b in zip(inst, done_b))
        vec = sum(2 * l_b * 5 * 8 * s_.n for s_, l_b in zip(inst, done_b))
        alg = (basis + vec) / (2 * L)
        peak_hbm = measured_peaks().get("hbm_gbs", 6801.7)
        gbs = alg / (half_ms / 1e3) / 1e9
        tflops = 2 * fma / (half_ms / 1e3) / 1e12
        kern = {"half_step_roofline": {
                    "kernel": "k_half_batch", "bound": "alu", "achieved": round(tflops, 4),
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": round(tflops / FP64_PEAK_TFLOPS, 4),
                    "traffic": None, "pipe": "fp64 (CGS2: 4 n M FMA per half-step)",
                    "peak_source": FP64_PEAK_SOURCE,
                    "avg_launch_ms": round(half_ms, 5), "launches_timed": int(ct["reorth_launches"]),
                    "algorithmic_per_launch": f"{fma:.4g} FP64 FMA, {alg:.4g} bytes (one read of each active "
                                              f"basis + vectors), averaged over the {2 * L} half-steps",
                    "hbm_achieved_gbs": round(gbs, 1), "hbm_frac": round(gbs / peak_hbm, 4),
                    "design_traffic_gbs": round((4 * basis + vec) / (2 * L) / (half_ms / 1e3) / 1e9, 1)},
                "batch_ms_graph_with_solve_and_u": round(ms / args.steps, 2),
                "batch_gkb_ms_graph": round(ms_graph_gkb, 2),
                "batch_gkb_ms_direct_timed": round(ms_direct, 2),
                "kernel_ms_sum": round(prod_ms + ct["reorth_ms"], 2),
                "products_ms": round(prod_ms, 2), "half_steps_ms": round(ct["reorth_ms"], 2),
                "timing": "a context with launch timing: the step loop launched directly, CUDA events around "
                          "each launch on the batch stream"}
    other = None
    if learned_arm:  # the same instances by the other forms, once each, for comparison
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record()
        one(False)
        g1.record()
        torch.cuda.synchronize()
        eg = errors()
        other = {"mixed_batched_gcv_hkt": {"ms": round(g0.elapsed_time(g1), 2),
                                           "re_median": float(np.median(eg)), "re_max": float(np.max(eg))},
                 "learned_err_not_worse_than_batched_gcv_frac":
                     float(np.mean(np.array(errs) <= 1.05 * np.array(eg)))}
        for name, prec, storage in (("fp64_single_gcv_hkt", R.RBF_FP64, R.RBF_ASSEMBLED),
                                    ("mixed_single_gcv_hkt", R.RBF_MIXED, R.RBF_MATRIX_FREE)):
            ms_sum, es = 0.0, []
            for b, s_ in enumerate(inst):
                n_b = s_.n
                nodes_b = torch.as_tensor(s_.soa(), device=dev)
                f_b = torch.as_tensor(fs[b], device=dev)
                P_b = torch.as_tensor(np.ascontiguousarray(pts[b].T), device=dev)
                A_b, lda_b = None, 0
                if storage == R.RBF_ASSEMBLED:
                    lda_b = R.padded_lda(n_b, prec)
                    A_b = torch.empty((n_b, lda_b), dtype=torch.float64, device=dev)
                op_b = ctx.rbf_operator_init(nodes_b, n_b, s_.n_interior, s_.params["c"], s_.params["k"], storage,
                                             prec, R.RBF_FORM_C, A_b, lda_b)
                st_b, *_ = R.make_state(torch, n_b, L, dev)
                c_b = torch.empty(n_b, dtype=torch.float64, device=dev)
                u_b = torch.empty(m, dtype=torch.float64, device=dev)
                torch.cuda.synchronize()
                h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                h0.record()
                if A_b is not None:
                    ctx.rbf_assemble(op_b)
                ctx.rbf_gkb(op_b, f_b, L, st_b)
                ctx.rbf_hkt(st_b, R.RBF_GCV, 0.0, c_b)
                ctx.rbf_evaluate(op_b, c_b, P_b, m, u_b)
                h1.record()
                torch.cuda.synchronize()
                ms_sum += h0.elapsed_time(h1)
                ue = w.plane_wave(pts[b], s_.params["k"], s_.params["d"])
                es.append(float(np.max(np.abs(u_b.cpu().numpy() - ue)) / np.max(np.abs(ue))))
                del A_b, op_b, st_b
            other[name] = {"ms": round(ms_sum, 2), "re_median": float(np.median(es)), "re_max": float(np.max(es))}
    ctx.close()
    if rank != 0:
        return None
    value = instances_all / (ms / 1e3)
    name = "batch96-learned" if learned_arm else "batch96"
    return {"metric": ("batched learned-stop HKT instances/s (96 uneven instances, at most 150 GKB steps each)"
                       if learned_arm else "batched HKT instances/s (96 uneven instances, 150 GKB steps each)"),
            "value": round(value, 3),
            "unit": "instances/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms / args.steps, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": name, "instances": len(inst), "rows_total": T, "gkb_steps": L,
                       "precision": "mixed", "storage": "matrix_free",
                       "rule": "learned (GCV fallback)" if learned_arm else "gcv", "test_points_per_instance": m},
            "mean_gkb_steps_per_instance": round(mean_steps, 2), "comparison": other,
            "gkb_steps_per_s": round(steps_total / (ms / 1e3), 1),
            "regenerated_entries_per_s": entries / (ms / 1e3),
            "re_vs_exact": {"median": float(np.median(errs)), "max": float(np.max(errs))},
            "roofline": roof,
            "e2e": {"value": round(inst_e2e / (ms_e2e / 1e3), 3), "unit": "instances/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": round(ms_e2e / args.steps, 2)},
            "gpu_launches": int(cnt["launches"]),
            "tuning": tune, "clocks": clocks, "kernel_times": kern,
            "cpu_baseline": None if args.no_cpu_baseline else cpu_baseline_batch(inst, fs, pts, L)}


# --------------------------------------------------------------------------- learned stop (pump casing)
def run_learned(args, rank, world, local_rank):
    """Pump-casing-like domain, N = 40000 (8000 surface + 32000 interior
    nodes), c = 0.1, k = 8, u at 2000 points.  The exact solution is the
    casing example's Gaussian exp(-|X|^2 / 10) (Sec. 5, Example 3); the plane
    wave along (1,1,1)/sqrt 3 is reported beside it.  One bench step = one
    learned-stop HKT solve through the C ABI: mixed precision (FP32
    matrix-free products, FP64 elsewhere), GKB for 10 steps, network forward,
    GKB resumed to the predicted l (at most 150), projected solve at the
    predicted lambda (GCV-HKT at 150 steps when rejected), reconstruction.
    Beside it, timed once per field: the learned stop, mixed GCV-HKT(150), and
    the plain FP64 assembled HKT(150) with GCV and with the L-curve."""
    import numpy as np
    import torch

    import workloads as w
    from paper_2511_09798_gb300 import learned
    from paper_2511_09798_gb300 import rbfkr as R

    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    ns = w.preset("pump40000")
    c, k, L = ns.params["c"], ns.params["k"], ns.params["steps"]
    n = ns.n
    Pn = w.test_points(ns)
    m = Pn.shape[0]
    fields = {
        "gauss_sigma10": (w.gaussian_rhs(ns, 10.0, k), w.gaussian(Pn, 10.0)),
        "plane_wave": (w.plane_wave_rhs(ns, k), w.plane_wave(Pn, k)),
    }
    stream = torch.cuda.current_stream()
    ctx = R.Context(local_rank, stream=stream, timing=2)
    net = learned.StopNet.load(torch, os.path.join(ROOT, "paper_2511_09798_gb300", "stopnet_weights.npz"),
                               device=dev)
    snet = net.c_struct()
    f_np, ue = fields["gauss_sigma10"]
    nodes_h = torch.from_numpy(ns.soa()).pin_memory()
    pts_h = torch.from_numpy(np.ascontiguousarray(Pn.T)).pin_memory()
    f_h = torch.from_numpy(f_np).pin_memory()
    nodes_d, pts_d, f_d = nodes_h.to(dev), pts_h.to(dev), f_h.to(dev)
    st, *_ = R.make_state(torch, n, L, dev)
    coef = torch.empty(n, dtype=torch.float64, device=dev)
    u_d = torch.empty(m, dtype=torch.float64, device=dev)
    u_h = torch.empty(m, dtype=torch.float64).pin_memory()
    op = ctx.rbf_operator_init(nodes_d, n, ns.n_interior, c, k, R.RBF_MATRIX_FREE, R.RBF_MIXED)
    infos = []

    def rel_err(u_exact):
        return float(np.max(np.abs(u_d.cpu().numpy() - u_exact)) / np.max(np.abs(u_exact)))

    def one_step(f, e2e=False):
        if e2e:
            nodes_d.copy_(nodes_h, non_blocking=True)
            pts_d.copy_(pts_h, non_blocking=True)
            f_d.copy_(f_h, non_blocking=True)
        info = ctx.rbf_learned_hkt(op, f, snet, st, coef)
        ctx.rbf_evaluate(op, coef, pts_d, m, u_d)
        if e2e:
            u_h.copy_(u_d, non_blocking=True)
        infos.append(info)
        return info.steps

    def timed(k_steps, e2e):
        rank_barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        done = sum(one_step(f_d, e2e) for _ in range(k_steps))
        e1.record(stream)
        torch.cuda.synchronize()
        return reduce_over_ranks(e0.elapsed_time(e1), done, dev)

    for _ in range(args.warmup):
        one_step(f_d)
    ctx.rbf_get_counters(reset=True)
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
    ms, done = timed(args.steps, False)
    clocks = sampler.stop() if sampler else None
    cnt = ctx.rbf_get_counters(reset=True)
    err_learned = rel_err(ue)
    last = infos[-1]
    ms_e2e, _ = timed(args.steps, True)

    def arm(f, u_exact, prec, storage, rule):
        A = None
        lda = 0
        if storage == R.RBF_ASSEMBLED:
            lda = R.padded_lda(n, prec)
            A = torch.empty((n, lda), dtype=torch.float64, device=dev)
        o = ctx.rbf_operator_init(nodes_d, n, ns.n_interior, c, k, storage, prec, R.RBF_FORM_C, A, lda)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if rule == "learned":
            info = ctx.rbf_learned_hkt(o, f, snet, st, coef)
            lam, s1 = info.solve.lambda_, info.solve.sigma1
        else:
            if A is not None:
                ctx.rbf_assemble(o)
            ctx.rbf_gkb(o, f, L, st)
            info = ctx.rbf_hkt(st, rule, 0.0, coef)
            lam, s1 = info.lambda_, info.sigma1
        ctx.rbf_evaluate(o, coef, pts_d, m, u_d)
        e1.record(stream)
        torch.cuda.synchronize()
        out = {"ms": round(e0.elapsed_time(e1), 2), "max_err_vs_exact": rel_err(u_exact),
               "gkb_steps": st.steps_done, "t": float(np.log10(lam / s1)) if lam > 0 and s1 > 0 else None}
        if rule == "learned":
            out.update({"accepted": info.accepted, "l_pred": info.l_pred, "t_pred": info.t_pred})
        del A, o
        return out

    arms = {}
    for name, (f_np2, u_ex) in fields.items():
        f2 = torch.as_tensor(f_np2, device=dev)
        arms[name] = {"learned_mixed_mf": arm(f2, u_ex, R.RBF_MIXED, R.RBF_MATRIX_FREE, "learned"),
                      "mixed_mf_gcv_hkt": arm(f2, u_ex, R.RBF_MIXED, R.RBF_MATRIX_FREE, R.RBF_GCV),
                      "fp64_assembled_gcv_hkt": arm(f2, u_ex, R.RBF_FP64, R.RBF_ASSEMBLED, R.RBF_GCV),
                      "fp64_assembled_lcurve_hkt": arm(f2, u_ex, R.RBF_FP64, R.RBF_ASSEMBLED, R.RBF_LCURVE)}
    ctx.close()
    if rank != 0:
        return None
    p_ms, p_cnt = cnt["product_ms"], cnt["product_launches"]
    avg_ms = (p_ms[0] + p_ms[1]) / max(1, p_cnt[0] + p_cnt[1])
    roof = mf_roofline(n, ns.n_interior, avg_ms)
    roof.update({"kernel": "matrix-free FP32 products (p = A z, r = A^T w)", "avg_launch_ms": round(avg_ms, 5),
                 "launches_timed": int(p_cnt[0] + p_cnt[1]), "algorithmic_per_launch": f"{n * n} entries"})
    solves = args.steps * world
    value = solves / (ms / 1e3)
    ms_solve = ms / args.steps
    base = arms["gauss_sigma10"]["fp64_assembled_gcv_hkt"]
    return {"metric": METRIC, "value": round(value, 3), "unit": "HKT solutions/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_solve, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": "pump40000-learned", "n": n, "n_interior": ns.n_interior, "c": c, "k": k,
                       "exact_solution": "exp(-|X|^2/10)", "l_max": L, "precision": "mixed",
                       "storage": "matrix_free", "rule": "learned (GCV fallback)", "test_points": m,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (node set and Krylov bases streamed each product)"},
            "time_to_solution_ms": round(ms_solve, 2),
            "learned": {"gkb_steps": last.steps, "l_pred": last.l_pred, "t_pred": last.t_pred,
                        "accepted": last.accepted, "in_distribution": last.in_distribution,
                        "max_err_vs_exact": err_learned},
            "comparison_single_runs": arms,
            "speedup_vs_fp64_gcv_hkt": round(base["ms"] / ms_solve, 2),
            "roofline": roof,
            "e2e": {"value": round(solves / (ms_e2e / 1e3), 3), "unit": "HKT solutions/s",
                    "h2d_bytes_per_step": (nodes_h.numel() + pts_h.numel() + f_h.numel()) * 8,
                    "d2h_bytes_per_step": u_h.numel() * 8, "ms_per_step": round(ms_e2e / args.steps, 2)},
            "gpu_launches": int(cnt["launches"]),
            "cpu_baseline": None if args.no_cpu_baseline else cpu_baseline_rows(ns, c, k, L),
            "clocks": clocks}


# --------------------------------------------------------------------------- paper-shaped sweep
def run_paper_sweep(args, rank, world, local_rank):
    """Stand-in for the accuracy tables of the cube and sphere examples (Sec.
    5, Examples 1 and 2; their Gmsh nodes are not available): the Gaussian
    exp(-|X - X0|^2 / 20) (X0 = 0 in the cube, (0.25, 0.25, 0) in the ball),
    k = 3, c = 2 (the shape parameter is not printed; c = 2 gives kappa(A) of
    the printed order at N = 359), random / uniform / Halton nodes at N ~ 359,
    2154, 6511, FP64 assembled.  Per case: full-SVD Tikhonov with GCV
    (Tikh-Rg), Ine-TSVD and HKT on 140 (cube) or 180 (sphere) GKB steps with
    GCV, HKT with the L-curve, each timed on the device from the assembled
    operator to u at 2000 points, with Re = max|u - u_exact| / max|u_exact|."""
    import numpy as np
    import torch

    import workloads as w
    from paper_2511_09798_gb300 import rbfkr as R
    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    stream = torch.cuda.current_stream()
    ctx = R.Context(local_rank, stream=stream)
    c, k, sigma = 2.0, 3.0, 20.0
    rows = []
    t_all = 0.0
    for dom, L, center in (("cube", 140, (0.0, 0.0, 0.0)), ("sphere", 180, (0.25, 0.25, 0.0))):
        for dist in ("random", "uniform", "halton"):
            for n_target in (359, 2154, 6511):
                ns = w.paper_nodes(dom, dist, n_target, w.nodes.BASE_SEED + 700 + n_target)
                n = ns.n
                P = w.test_points(ns, 2000, seed=w.nodes.BASE_SEED + 1700 + n_target)
                ue = w.gaussian(P, sigma, center)
                f = torch.as_tensor(w.gaussian_rhs(ns, sigma, k, center), device=dev)
                nodes = torch.as_tensor(ns.soa(), device=dev)
                pts = torch.as_tensor(np.ascontiguousarray(P.T), device=dev)
                lda = R.padded_lda(n, R.RBF_FP64)
                A = torch.empty((n, lda), dtype=torch.float64, device=dev)
                op = ctx.rbf_operator_init(nodes, n, ns.n_interior, c, k, R.RBF_ASSEMBLED, R.RBF_FP64, A=A, lda=lda)
                st, *_ = R.make_state(torch, n, L, dev)
                coef = torch.empty(n, dtype=torch.float64, device=dev)
                u = torch.empty(2000, dtype=torch.float64, device=dev)
                row = {"domain": dom, "nodes": dist, "n": n}

                def timed(name, fn):
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ctx.rbf_assemble(op)
                    fn()
                    ctx.rbf_evaluate(op, coef, pts, 2000, u)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1)
                    err = float(np.max(np.abs(u.cpu().numpy() - ue)) / np.max(np.abs(ue)))
                    row[name] = {"re": err, "ms": round(ms, 2)}
                    return ms

                t_all += timed("tikh_rg", lambda: ctx.rbf_tikhonov(op, f, R.RBF_GCV, 0.0, coef))
                t_all += timed("ine_tsvd", lambda: (ctx.rbf_gkb(op, f, L, st), ctx.rbf_ine_tsvd(st, 0, coef)))
                t_all += timed("hkt_gcv", lambda: (ctx.rbf_gkb(op, f, L, st), ctx.rbf_hkt(st, R.RBF_GCV, 0.0, coef)))
                t_all += timed("hkt_lcurve",
                               lambda: (ctx.rbf_gkb(op, f, L, st), ctx.rbf_hkt(st, R.RBF_LCURVE, 0.0, coef)))
                rows.append(row)
                del A, st, op
    ctx.close()
    if rank != 0:
        return None
    return {"metric": "paper-shaped accuracy sweep: Re and device time per method", "value": round(t_all / 1e3, 3),
            "unit": "device seconds for the sweep", "n_gpus": world, "steps": 1, "warmup": 0,
            "ms_per_step": round(t_all, 1), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "paper-sweep", "c": c, "k": k, "sigma": sigma,
                       "gkb_steps": {"cube": 140, "sphere": 180}, "test_points": 2000},
            "rows": rows}


# --------------------------------------------------------------------------- matrix-free product roofline
def mf_product_roofline(local_rank, steps=80):
    """The matrix-free FP32 product (entries regenerated from the node
    coordinates) on the 20 000-node sphere (c = 0.15, k = 10): the library's
    product timing (CUDA events around every product launch on the launching
    stream) over a GKB run of `steps` steps after a 20-step warm-up run, as
    regenerated entries per second and a fraction of the FP32 pipe (the
    operations of mf_pair_ops: each node pair evaluated once for A_ij and A_ji,
    the MUFU rsqrt beside them)."""
    import torch

    import workloads as w
    from paper_2511_09798_gb300 import rbfkr as R
    ns = w.preset("sphere20000")
    n = ns.n
    dev = f"cuda:{local_rank}"
    ctx = R.Context(local_rank, stream=torch.cuda.current_stream(), timing=2)
    nodes = torch.as_tensor(ns.soa(), device=dev)
    op = ctx.rbf_operator_init(nodes, n, ns.n_interior, 0.15, 10.0, R.RBF_MATRIX_FREE, R.RBF_MIXED)
    f = torch.as_tensor(w.plane_wave_rhs(ns, 10.0), device=dev)
    ctx.rbf_gkb(op, f, 20, R.make_state(torch, n, 20, dev)[0])  # warm-up
    torch.cuda.synchronize()
    ctx.rbf_get_counters(reset=True)
    ctx.rbf_gkb(op, f, steps, R.make_state(torch, n, steps, dev)[0])
    torch.cuda.synchronize()
    cnt = ctx.rbf_get_counters(reset=True)
    ctx.close()
    launches = int(sum(cnt["product_launches"]))
    ms = sum(cnt["product_ms"]) / max(1, launches)
    roof = mf_roofline(n, ns.n_interior, ms)
    roof.update({"kernel": "k_mf_sym (FP32 matrix-free product, sphere20000)", "avg_launch_ms": round(ms, 5),
                 "launches_timed": launches,
                 "timing": f"CUDA events around each product launch (k_mf_sym and its slot fold) of a "
                           f"{steps}-step GKB run"})
    return roof


# --------------------------------------------------------------------------- forms at equal error
def forms_comparison(local_rank, count=24, L=150, m=500, reps=1):
    """Time to solution and error against the exact solution of the same
    uneven instances by each form of the method: plain FP64 HKT (assembled,
    one instance after another, and all instances on concurrent lanes), mixed
    precision (FP32 matrix-free products, FP64 elsewhere; one after another
    and on lanes), the batched mixed form, and the batched mixed form with the
    learned stop (GCV fallback).

    Instances: the held-out draws of the learned stop's generator (cube or
    sphere, N ~ U{2000..16000}, c log-uniform in [0.05, 1], k ~ U[1, 20]) with
    the paper's Gaussian exact solution exp(-|X - X0|^2 / sigma) (sigma
    log-uniform in [0.05, 10]): fields HKT resolves, so equal error is a real
    test (plane waves at k up to 20 are not resolved by 150 GKB steps).  All
    GKB runs take L steps (the learned stop fewer); rule GCV; u at m test
    points per instance; device time by CUDA events around each form."""
    import numpy as np
    import torch

    import workloads as w
    from paper_2511_09798_gb300 import learned
    from paper_2511_09798_gb300 import rbfkr as R
    dev = f"cuda:{local_rank}"
    inst = w.stop_instances(count, 2000, 16000, seed0=w.nodes.BASE_SEED + 50000, gauss_share=1.0)
    fs = [w.instance_rhs(s_) for s_ in inst]
    pts = [w.test_points(s_, m, seed=s_.params["seed"] + 7) for s_ in inst]
    ue = [w.instance_field(s_, P) for s_, P in zip(inst, pts)]
    stream = torch.cuda.current_stream()
    ctx = R.Context(local_rank, stream=stream)
    nodes = [torch.as_tensor(s_.soa(), device=dev) for s_ in inst]
    f_d = [torch.as_tensor(f, device=dev) for f in fs]
    P_d = [torch.as_tensor(np.ascontiguousarray(P.T), device=dev) for P in pts]
    u_d = [torch.empty(m, dtype=torch.float64, device=dev) for _ in inst]
    coefs = [torch.empty(s_.n, dtype=torch.float64, device=dev) for s_ in inst]

    def errs():
        return [float(np.max(np.abs(u.cpu().numpy() - e)) / np.max(np.abs(e))) for u, e in zip(u_d, ue)]

    def timed(fn):
        fn()  # warm-up (workspace, tuning, graph capture)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, errs()

    out = {}
    # plain FP64, assembled, one instance after another
    mats = [torch.empty((s_.n, R.padded_lda(s_.n, R.RBF_FP64)), dtype=torch.float64, device=dev) for s_ in inst]
    ops64 = [ctx.rbf_operator_init(nd, s_.n, s_.n_interior, s_.params["c"], s_.params["k"], R.RBF_ASSEMBLED,
                                   R.RBF_FP64, R.RBF_FORM_C, A, A.shape[1]) for nd, s_, A in zip(nodes, inst, mats)]
    sts = [R.make_state(torch, s_.n, L, dev)[0] for s_ in inst]

    def fp64_serial():
        for b in range(count):
            ctx.rbf_assemble(ops64[b])
            ctx.rbf_gkb(ops64[b], f_d[b], L, sts[b])
            ctx.rbf_hkt(sts[b], R.RBF_GCV, 0.0, coefs[b])
            ctx.rbf_evaluate(ops64[b], coefs[b], P_d[b], m, u_d[b])

    def fp64_lanes():
        ctx.rbf_gkb_many(ops64, f_d, L, sts, assemble=True)
        ctx.rbf_hkt_many(sts, R.RBF_GCV, 0.0, coefs)
        for b in range(count):
            ctx.rbf_evaluate(ops64[b], coefs[b], P_d[b], m, u_d[b])

    out["fp64_single"] = timed(fp64_serial)
    out["fp64_lanes"] = timed(fp64_lanes)
    del mats, ops64
    torch.cuda.empty_cache()
    opsm = [ctx.rbf_operator_init(nd, s_.n, s_.n_interior, s_.params["c"], s_.params["k"], R.RBF_MATRIX_FREE,
                                  R.RBF_MIXED) for nd, s_ in zip(nodes, inst)]

    def mixed_serial():
        for b in range(count):
            ctx.rbf_gkb(opsm[b], f_d[b], L, sts[b])
            ctx.rbf_hkt(sts[b], R.RBF_GCV, 0.0, coefs[b])
            ctx.rbf_evaluate(opsm[b], coefs[b], P_d[b], m, u_d[b])

    def mixed_lanes():
        ctx.rbf_gkb_many(opsm, f_d, L, sts)
        ctx.rbf_hkt_many(sts, R.RBF_GCV, 0.0, coefs)
        for b in range(count):
            ctx.rbf_evaluate(opsm[b], coefs[b], P_d[b], m, u_d[b])

    out["mixed_single"] = timed(mixed_serial)
    out["mixed_lanes"] = timed(mixed_lanes)
    bt, keep = R.make_batch(torch, inst, [s_.params["c"] for s_ in inst], [s_.params["k"] for s_ in inst], fs, L, dev)
    T = int(keep["offsets"][-1])
    coef_b = torch.empty(T, dtype=torch.float64, device=dev)
    P_all = torch.as_tensor(np.concatenate([P.T.ravel() for P in pts]), device=dev)
    u_all = torch.empty(m * count, dtype=torch.float64, device=dev)

    def scatter():
        for b in range(count):
            u_d[b].copy_(u_all[b * m:(b + 1) * m])

    def mixed_batched():
        ctx.rbf_batch_gkb(bt, L)
        ctx.rbf_batch_hkt(bt, R.RBF_GCV, coef_b)
        ctx.rbf_batch_evaluate(bt, coef_b, P_all, [m] * count, u_all)
        scatter()

    out["mixed_batched"] = timed(mixed_batched)
    net = learned.StopNet.load(torch, os.path.join(ROOT, "paper_2511_09798_gb300", "stopnet_weights.npz"), device=dev)
    snet = net.c_struct()
    steps_learned = []

    def mixed_batched_learned():
        ctx.rbf_batch_learned_hkt(bt, snet, coef_b)
        ctx.rbf_batch_evaluate(bt, coef_b, P_all, [m] * count, u_all)
        scatter()
        steps_learned[:] = [bt.steps_done[b] for b in range(count)]

    out["mixed_batched_learned"] = timed(mixed_batched_learned)
    ctx.close()
    ref = np.array(out["fp64_single"][1])
    res = {}
    for name, (ms, e) in out.items():
        e = np.array(e)
        res[name] = {"ms": round(ms, 2), "ms_per_instance": round(ms / count, 3),
                     "re_median": float(np.median(e)), "re_q90": float(np.quantile(e, 0.9)),
                     "re_max": float(np.max(e)),
                     "err_not_worse_than_fp64_frac": float(np.mean(e <= 1.05 * ref)),
                     "speedup_vs_fp64_single": round(out["fp64_single"][0] / ms, 2)}
    res["mixed_batched_learned"]["mean_gkb_steps"] = float(np.mean(steps_learned))
    return {"instances": count, "gkb_steps": L, "exact": "Gaussian exp(-|X - X0|^2 / sigma)", "rule": "gcv",
            "test_points_per_instance": m, "n_range": [min(s_.n for s_ in inst), max(s_.n for s_ in inst)],
            "forms": res}


# --------------------------------------------------------------------------- FP64 pipe probe
def run_fp64_probe(args, rank, world, local_rank):
    """Measured FP64 throughput of this GPU (the peak the FP64 products are
    reported against): FP64 FMA alone, FP64 MMA (mma.sync m8n8k4) alone, and
    both issued by every warp, each on one resident wave of CTAs for about
    0.5 s, with the SM clock sampled by nvidia-smi during the runs."""
    import torch

    from paper_2511_09798_gb300 import rbfkr as R
    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    ctx = R.Context(local_rank, stream=torch.cuda.current_stream())
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    scratch = torch.empty(sms * 8 * 256, dtype=torch.float64, device=dev)
    names = {0: "fp64_fma", 1: "fp64_mma_m8n8k4", 2: "fma_and_mma"}
    out = {}
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
    for mode in (0, 1, 2):
        iters = 1 << 12
        ms, fl = ctx.rbf_probe_fp64(mode, iters, scratch)  # warm-up and size
        iters = max(1, int(iters * 500.0 / max(ms, 1e-3)))
        best = None
        for _ in range(3):
            ms, fl = ctx.rbf_probe_fp64(mode, iters, scratch)
            if best is None or ms < best[0]:
                best = (ms, fl)
        out[names[mode]] = {"tflops": round(best[1] / (best[0] / 1e3) / 1e12, 4), "ms": round(best[0], 2),
                            "iters": iters}
    clocks = sampler.stop() if sampler else None
    ctx.close()
    if rank != 0:
        return None
    mhz = clocks["sm_mhz"] if clocks else 2070.0
    for v in out.values():
        v["flop_per_clk_per_sm"] = round(v["tflops"] * 1e12 / (sms * mhz * 1e6), 3)
    fma = out["fp64_fma"]
    return {"metric": "FP64 pipe throughput (roofline peak of the FP64 products)", "value": fma["tflops"],
            "unit": "TFLOP/s", "n_gpus": 1, "steps": 3, "warmup": 1, "ms_per_step": fma["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "fp64-pipe-probe", "sms": sms}, "probes": out,
            "fma_per_clk_per_sm": round(fma["flop_per_clk_per_sm"] / 2, 3), "clocks": clocks}


# --------------------------------------------------------------------------- oracle
def oracle_solve(wl, c, k, steps):
    from oracle import evaluate as OE
    from oracle import gkb as OG
    from oracle import mq as OM
    from oracle import regularize as OR
    ns = wl["ns"]
    A = OM.assemble(ns.X, ns.n_interior, c, k)
    g = OG.gkb(A, None, wl["fs"][k], steps)
    h = OR.hkt(g, "gcv")
    OE.reconstruct(h["coef"], ns.X, wl["points"], c)
    return g.steps_done


def host_info():
    """Host threads the NumPy oracle uses, CPU model and BLAS build (for the CPU baseline)."""
    import numpy as np
    threads = None
    try:
        from threadpoolctl import threadpool_info
        blas = [d for d in threadpool_info() if d.get("user_api") == "blas"]
        if blas:
            threads = int(blas[0]["num_threads"])
    except Exception:
        pass
    if threads is None:
        env = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS")
        threads = int(env) if env and env.isdigit() else os.cpu_count()
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    if key == "model name":
                        break
    except OSError:
        pass
    import platform
    model = f"{platform.machine()} {model}" if model else platform.machine()
    try:
        b = np.show_config(mode="dicts")["Build Dependencies"]["blas"]
        blas_name = f"{b.get('name')} {b.get('version')}"
    except Exception:
        blas_name = "unknown"
    return {"cores": threads, "cpu": model, "blas": blas_name}


def cpu_baseline_batch(inst, fs, pts, steps, budget_s=15.0):
    """The oracle on the batch's instances in order (each one a full FP64
    solve: assemble, GKB, HKT with GCV, u at the test points) until budget_s
    has passed; instances/s over that sample."""
    from oracle import evaluate as OE
    from oracle import gkb as OG
    from oracle import mq as OM
    from oracle import regularize as OR
    t0 = time.perf_counter()
    count, rows = 0, 0
    for b, s_ in enumerate(inst):
        c, k = s_.params["c"], s_.params["k"]
        A = OM.assemble(s_.X, s_.n_interior, c, k)
        g = OG.gkb(A, None, fs[b], steps)
        h = OR.hkt(g, "gcv")
        OE.reconstruct(h["coef"], s_.X, pts[b], c)
        del A, g, h
        count += 1
        rows += s_.n
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    hi = host_info()
    return {"value": round(count / dt, 4), "unit": "instances/s", "cores": hi["cores"], "kind": "oracle",
            "cpu": hi["cpu"], "blas": hi["blas"],
            "sample": f"the first {count} of {len(inst)} instances ({rows} rows in all), each a full FP64 solve "
                      f"(assemble, {steps} GKB steps, SVD, GCV, lift, u at {pts[0].shape[0]} points): {dt:.1f} s"}


def cpu_baseline_rows(ns, c, k, steps, rows=1000, sample_steps=10):
    """CPU baseline for a workload whose FP64 matrix is too large for the host
    oracle: the oracle's operations on a sample of the same matrix, scaled to
    one full FP64 GCV-HKT(steps) solve.  Timed: assembling `rows` rows of A
    (oracle entry formulas), `sample_steps` pairs of products with that row
    block, and `sample_steps` two-pass Gram-Schmidt steps against a basis of
    steps / 2 vectors of length N (the average basis size).  Scaled: assembly
    and products by N / rows, products and Gram-Schmidt by steps / sample_steps
    (two Gram-Schmidt calls per GKB step); the projected SVD, the lambda sweep
    and u are left out (milliseconds)."""
    import numpy as np

    from oracle import mq as OM
    n = ns.n
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    D = OM.distances(ns.X[:rows], ns.X)
    blk = np.empty_like(D)
    ri = min(rows, ns.n_interior)
    blk[:ri] = OM.lphi(D[:ri], c, k)
    blk[ri:] = OM.phi(D[ri:], c)
    t_asm = time.perf_counter() - t0
    z = rng.standard_normal(n)
    t0 = time.perf_counter()
    for _ in range(sample_steps):
        y = blk @ z
        z = blk.T @ y
        z /= np.linalg.norm(z)
    t_prod = time.perf_counter() - t0
    Q, _ = np.linalg.qr(rng.standard_normal((n, max(1, steps // 2))))
    v = rng.standard_normal(n)
    t0 = time.perf_counter()
    for _ in range(sample_steps):
        for _ in range(2):
            v = v - Q @ (Q.T @ v)
    t_gs = time.perf_counter() - t0
    scale_rows = n / rows
    t_full = t_asm * scale_rows + t_prod * scale_rows * steps / sample_steps + t_gs * 2 * steps / sample_steps
    hi = host_info()
    return {"value": round(1.0 / t_full, 5), "unit": "HKT solutions/s", "cores": hi["cores"], "kind": "oracle",
            "cpu": hi["cpu"], "blas": hi["blas"],
            "sample": (f"scaled from a sample: oracle assembly of {rows} of {n} rows ({t_asm:.2f} s), "
                       f"{sample_steps} product pairs with that block ({t_prod:.2f} s) and {sample_steps} "
                       f"Gram-Schmidt steps against {max(1, steps // 2)} vectors ({t_gs:.2f} s), scaled to one "
                       f"FP64 GCV-HKT({steps}) solve: {t_full:.1f} s")}


def cpu_baseline(wl, sample_steps):
    if wl["ns"].n > 10000:
        sample_steps = min(sample_steps, 10)
    c, k = wl["cases"][0]
    t0 = time.perf_counter()
    done = oracle_solve(wl, c, k, sample_steps)
    dt = time.perf_counter() - t0
    hi = host_info()
    return {"value": round(done / dt, 3), "unit": "GKB steps/s", "cores": hi["cores"], "kind": "oracle",
            "cpu": hi["cpu"], "blas": hi["blas"],
            "sample": f"one full solve (assemble, {sample_steps} GKB steps, SVD, GCV, lift, u at "
                      f"{wl['points'].shape[0]} points) of {wl['name']} at c={c}, k={k}: {dt:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    wl = workload(args.workload)
    L = wl["steps"]
    c, k = wl["cases"][0]
    for _ in range(args.warmup):
        oracle_solve(wl, c, k, L)
    t0 = time.perf_counter()
    done = 0
    for _ in range(args.steps):
        done += oracle_solve(wl, c, k, L)
    dt = time.perf_counter() - t0
    v = round(done / dt, 3)
    return {"metric": METRIC, "value": v, "unit": "GKB steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": wl["name"], "n": wl["ns"].n, "gkb_steps": L, "cases_c_k": [(c, k)],
                       "solves_per_step": 1, "precision": "fp64", "storage": "assembled", "rule": "gcv"},
            "cpu_baseline": {"value": v, "unit": "GKB steps/s", **host_info(), "kind": "oracle",
                             "sample": f"one full solve of {wl['name']} at c={c}, k={k} per step"},
            "e2e": {"value": v, "unit": "GKB steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def single_solve(args):
    import torch

    from paper_2511_09798_gb300 import rbfkr as R
    wl = workload(args.workload)
    ns, (c, k), L = wl["ns"], wl["cases"][0], wl["steps"]
    prec = R.RBF_FP64 if wl["precision"] == "fp64" else R.RBF_MIXED
    storage = R.RBF_ASSEMBLED if wl["storage"] == "assembled" else R.RBF_MATRIX_FREE
    ctx = R.Context(0, fma_products=int(args.fma_products))
    n, m = ns.n, wl["points"].shape[0]
    nodes = torch.from_numpy(ns.soa()).cuda()
    pts = torch.from_numpy(wl["points"].T.copy()).cuda()
    f = torch.from_numpy(wl["fs"][k]).cuda()
    lda = R.padded_lda(n, prec)
    A = None
    if storage == R.RBF_ASSEMBLED:
        A = torch.empty((n, lda), dtype=torch.float64 if prec == R.RBF_FP64 else torch.float32, device="cuda")
    st, *_ = R.make_state(torch, n, L)
    coef = torch.empty(n, dtype=torch.float64, device="cuda")
    u = torch.empty(m, dtype=torch.float64, device="cuda")
    op = ctx.rbf_operator_init(nodes, n, ns.n_interior, c, k, storage, prec, R.RBF_FORM_C, A,
                               lda if A is not None else 0)
    if A is not None:
        ctx.rbf_assemble(op)
    ctx.rbf_gkb(op, f, L, st)
    info = ctx.rbf_hkt(st, R.RBF_GCV, 0.0, coef)
    ctx.rbf_evaluate(op, coef, pts, m, u)
    torch.cuda.synchronize()
    print(json.dumps({"single_solve": wl["name"], "steps_done": st.steps_done, "lambda": info.lambda_,
                      "index": info.index, "launches": ctx.rbf_get_counters()["launches"]}))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cube8000")
    ap.add_argument("--lanes", type=int, default=0,
                    help="streams for the independent (c, k) solves of a step (0 = one per solve, 1 = serial)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the forms comparison of the default workload")
    ap.add_argument("--jsonl", default=None, help="also append the result line to this JSONL file")
    ap.add_argument("--single-solve", action="store_true",
                    help="run one untimed solve of the first case and exit (profiling target)")
    ap.add_argument("--fma-products", action="store_true",
                    help="FP64 assembled products with FP64 FMAs on A instead of the exact fixed-point copies")
    args = ap.parse_args()
    if args.single_solve:
        single_solve(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload in ("batch96", "batch96-learned"):
        out = run_batch(args, rank, world, local_rank)
    elif args.workload == "pump40000-learned":
        out = run_learned(args, rank, world, local_rank)
    elif args.workload == "paper-sweep":
        out = run_paper_sweep(args, rank, world, local_rank)
    elif args.workload == "fp64-pipe-probe":
        out = run_fp64_probe(args, rank, world, local_rank)
    elif args.workload == "forms-gauss":
        import torch
        torch.cuda.set_device(local_rank)
        t0 = time.perf_counter()
        fc = forms_comparison(local_rank)
        out = None if rank != 0 else {
            "metric": "time to HKT solution of 24 uneven Gaussian instances, per form", "value":
                fc["forms"]["mixed_batched_learned"]["speedup_vs_fp64_single"], "unit": "x plain FP64 HKT",
            "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": fc["forms"]["mixed_batched_learned"]["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic", "config": {"workload": "forms-gauss"}, "comparison": fc,
            "wall_s": round(time.perf_counter() - t0, 1)}
    else:
        out = run_ours(args, rank, world, local_rank)
        if out is not None and not args.no_cpu_baseline:
            wl = workload(args.workload)
            out["cpu_baseline"] = cpu_baseline(wl, wl["steps"])
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if out is not None:
        line = json.dumps(out)
        print(line, flush=True)
        if args.jsonl:
            with open(args.jsonl, "a") as fh:
                fh.write(line + "\n")


if __name__ == "__main__":
    main()
