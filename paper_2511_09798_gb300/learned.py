"""Learned stopping index and lambda for Hybrid Krylov-Tikhonov (Algorithm 4).

The paper runs a fixed number of GKB steps l and picks lambda on the projected
problem by GCV or the L-curve (Sec. 3.2-3.4); it leaves cheaper stopping to
future work (Sec. 6).  This module trains a small regressor that reads the
first 10 GKB steps (the 10 Ritz values of C_10 and the 10 least-squares
residual norms) and predicts ln l* and t* = log10(lambda* / s~_1), so that GKB
stops early and the lambda sweep is skipped.  Everything numeric runs in the
library's CUDA kernels through the C ABI: the batched GKB that generates the
training runs, the reconstruction of every Krylov vector at test points, the
error table over (l, lambda), the features, the network's forward and backward
passes and Adam.  Host code only arranges buffers, shuffles the sample order,
and turns the small error tables into labels.

Labels (the paper is silent; these are this module's readings):
  * E(l, t) = max-norm error of the HKT reconstruction against the known
    field at test points, for l in ``ells`` and t on the lambda grid;
  * l* = the smallest l whose best error min_t E(l, t) is within a factor
    (1 + rel_tol) of the best error over all l;
  * t* = the median of the grid points t whose error at l* is within the same
    factor of min_t E(l*, t) (the middle of the flat bottom, not an end of it).
"""
from __future__ import annotations

import math

import numpy as np

from . import rbfkr as R

FEAT_STEPS = 10
N_IN, N_HID, N_OUT = R.RBF_MLP_IN, R.RBF_MLP_HIDDEN, R.RBF_MLP_OUT
N_PARAMS = R.RBF_MLP_PARAMS


def init_params(seed: int = 0) -> np.ndarray:
    """Glorot-uniform weights, zero biases, in the library's parameter layout
    (W1 [20][128], b1, W2 [128][128], b2, W3 [128][2], b3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for fi, fo in ((N_IN, N_HID), (N_HID, N_HID), (N_HID, N_OUT)):
        a = math.sqrt(6.0 / (fi + fo))
        parts.append(rng.uniform(-a, a, size=fi * fo))
        parts.append(np.zeros(fo))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == N_PARAMS
    return p


class StopNet:
    """Trained parameters, standardisation and acceptance rules."""

    def __init__(self, torch, params, feat_mean, feat_std, out_mean, out_std, l_min=10, l_max=150,
                 window=5, accept_tol=math.inf, t_min=-16.0, t_max=0.0, fallback_rule=R.RBF_GCV, z_max=6.0,
                 device="cuda"):
        self.torch = torch
        self.params = torch.as_tensor(np.asarray(params, np.float32), device=device).contiguous()
        self.feat_mean = torch.as_tensor(np.asarray(feat_mean, np.float32), device=device).contiguous()
        self.feat_std = torch.as_tensor(np.asarray(feat_std, np.float32), device=device).contiguous()
        self.out_mean = np.asarray(out_mean, np.float32)
        self.out_std = np.asarray(out_std, np.float32)
        self.l_min, self.l_max, self.window = int(l_min), int(l_max), int(window)
        self.accept_tol, self.t_min, self.t_max = float(accept_tol), float(t_min), float(t_max)
        self.fallback_rule = int(fallback_rule)
        self.z_max = float(z_max)

    def c_struct(self) -> R.StopNet:
        s = R.StopNet()
        s.d_params = self.params.data_ptr()
        s.d_feat_mean = self.feat_mean.data_ptr()
        s.d_feat_std = self.feat_std.data_ptr()
        s.out_mean[0], s.out_mean[1] = float(self.out_mean[0]), float(self.out_mean[1])
        s.out_std[0], s.out_std[1] = float(self.out_std[0]), float(self.out_std[1])
        s.feat_steps = FEAT_STEPS
        s.l_min, s.l_max, s.window = self.l_min, self.l_max, self.window
        s.accept_tol, s.t_min, s.t_max = self.accept_tol, self.t_min, self.t_max
        s.fallback_rule = self.fallback_rule
        s.z_max = self.z_max
        return s

    def save(self, path: str) -> None:
        np.savez(path, params=self.params.cpu().numpy(), feat_mean=self.feat_mean.cpu().numpy(),
                 feat_std=self.feat_std.cpu().numpy(), out_mean=self.out_mean, out_std=self.out_std,
                 rules=np.array([self.l_min, self.l_max, self.window, self.fallback_rule], np.int64),
                 tols=np.array([self.accept_tol, self.t_min, self.t_max, self.z_max], np.float64))

    @classmethod
    def load(cls, torch, path: str, device="cuda", **override):
        z = np.load(path)
        kw = dict(l_min=int(z["rules"][0]), l_max=int(z["rules"][1]), window=int(z["rules"][2]),
                  fallback_rule=int(z["rules"][3]), accept_tol=float(z["tols"][0]), t_min=float(z["tols"][1]),
                  t_max=float(z["tols"][2]), z_max=float(z["tols"][3]))
        kw.update(override)
        return cls(torch, z["params"], z["feat_mean"], z["feat_std"], z["out_mean"], z["out_std"], device=device,
                   **kw)


def write_stopnet_file(npz_path: str, out_path: str) -> None:
    """Write a saved network (StopNet.save's .npz) in the library's binary
    layout, which rbf_stopnet_load reads from C: magic "RBFSTOP1"; int32 n_in,
    n_hidden, n_out, n_params, feat_steps; float32 params, feat_mean, feat_std,
    out_mean[2], out_std[2]; int32 l_min, l_max, window, fallback_rule;
    float64 accept_tol, t_min, t_max, z_max (little-endian)."""
    z = np.load(npz_path)
    rules = [int(x) for x in z["rules"]]
    with open(out_path, "wb") as fh:
        fh.write(b"RBFSTOP1")
        fh.write(np.array([N_IN, N_HID, N_OUT, N_PARAMS, FEAT_STEPS], "<i4").tobytes())
        for key in ("params", "feat_mean", "feat_std", "out_mean", "out_std"):
            fh.write(np.asarray(z[key], "<f4").tobytes())
        fh.write(np.array(rules, "<i4").tobytes())
        fh.write(np.asarray(z["tols"], "<f8").tobytes())


# --------------------------------------------------------------------------
# training runs and labels
# --------------------------------------------------------------------------

def label_runs(ctx, torch, node_sets, cs, ks, fs, points, urefs, L, ells, t_stride=4):
    """Run batched GKB (one graph launch, FP32 products) to L steps on every
    instance and return, per instance, the 10-step features [B][20] and the
    error table E [B][len(ells)][Jp] (inf where l exceeds the steps done).

    points[b]: test points (m_b x 3); urefs[b]: the known field there.
    """
    B = len(node_sets)
    bt, keep = R.make_batch(torch, node_sets, cs, ks, fs, L)
    ctx.rbf_batch_gkb(bt, L)
    off = keep["offsets"]
    J = ctx.grid_j
    Jp = (J - 1) // t_stride + 1
    feats = torch.empty((B, N_IN), dtype=torch.float32, device="cuda")
    E = np.full((B, len(ells), Jp), np.inf)
    for b in range(B):
        n = int(bt.n[b])
        st = batch_state_view(keep, bt, b, L)
        if st.steps_done < FEAT_STEPS:
            feats[b].fill_(float("nan"))
            continue
        ctx.rbf_stop_features(st, FEAT_STEPS, feats[b])
        op_nodes = keep["nodes"].data_ptr() + 8 * 3 * int(off[b])
        op = ctx.rbf_operator_init(op_nodes, n, int(bt.n_interior[b]), float(bt.c[b]), float(bt.k[b]),
                                   R.RBF_MATRIX_FREE, R.RBF_MIXED)
        P = np.ascontiguousarray(np.asarray(points[b], np.float64).T)
        m = P.shape[1]
        dP = torch.as_tensor(P, device="cuda")
        l_done = st.steps_done
        G = torch.empty((l_done, m), dtype=torch.float64, device="cuda")
        ctx.rbf_evaluate_many(op, st.d_Z, n, l_done, dP, m, G)
        uref = torch.as_tensor(np.asarray(urefs[b], np.float64), device="cuda")
        use = [e for e in ells if e <= l_done]
        if not use:
            continue
        err = torch.empty((len(use), Jp), dtype=torch.float64, device="cuda")
        ctx.rbf_hkt_error_table(st, G, m, m, uref, use, t_stride, err)
        E[b, :len(use)] = err.cpu().numpy()
    return feats.cpu().numpy(), E, np.array([bt.steps_done[b] for b in range(B)])


def batch_state_view(keep, bt, b, L) -> R.GkbState:
    """Single-instance GKB state viewing instance b of a batch's buffers."""
    n = int(bt.n[b])
    off = int(keep["offsets"][b])
    st = R.GkbState()
    st.d_W = keep["W"].data_ptr() + 8 * (L + 1) * off
    st.d_Z = keep["Z"].data_ptr() + 8 * L * off
    st.d_alpha = keep["alpha"].data_ptr() + 8 * L * b
    st.d_beta = keep["beta"].data_ptr() + 8 * (L + 1) * b
    st.ldw = st.ldz = n
    st.capacity, st.n = L, n
    st.steps_done, st.breakdown = bt.steps_done[b], bt.breakdown[b]
    return st


def grid_t(J: int, t_lo: float, t_hi: float, t_stride: int) -> np.ndarray:
    idx = np.arange(0, J, t_stride)
    step = (t_hi - t_lo) / (J - 1)
    t = idx * step + t_lo
    t[idx == J - 1] = t_hi
    return t


def make_labels(E, ells, tgrid, rel_tol=0.25):
    """(ln l*, t*) per instance from error tables E [B][n_ell][Jp]; rows with
    no finite entry get NaN."""
    B = E.shape[0]
    Y = np.full((B, 2), np.nan)
    for b in range(B):
        rowmin = np.min(E[b], axis=1)
        if not np.isfinite(rowmin).any():
            continue
        best = np.min(rowmin[np.isfinite(rowmin)])
        a = int(np.argmax(rowmin <= (1.0 + rel_tol) * best))
        row = E[b, a]
        ok = np.where(row <= (1.0 + rel_tol) * np.min(row))[0]
        Y[b, 0] = math.log(ells[a])
        Y[b, 1] = float(np.median(tgrid[ok]))
    return Y


# --------------------------------------------------------------------------
# training on the GPU
# --------------------------------------------------------------------------

def train(ctx, torch, X, Y, steps=3000, lr=1e-3, batch=256, seed=0, log_every=0, **rules):
    """Fit the network to standardised (X, Y) with Adam (the library's kernels).

    Returns (StopNet, losses).  Rows with any non-finite value are dropped.
    """
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    keep = np.all(np.isfinite(X), axis=1) & np.all(np.isfinite(Y), axis=1)
    X, Y = X[keep], Y[keep]
    fm, fs = X.mean(0), X.std(0)
    fs[fs < 1e-6] = 1.0
    om, os_ = Y.mean(0), Y.std(0)
    os_[os_ < 1e-6] = 1.0
    Xs = ((X - fm) / fs).astype(np.float32)
    Ys = ((Y - om) / os_).astype(np.float32)
    ns = Xs.shape[0]
    bs = min(batch, ns)
    params = torch.as_tensor(init_params(seed), device="cuda")
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    g = torch.zeros_like(params)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    losses = []
    t = 0
    while t < steps:
        perm = rng.permutation(ns)
        dX = torch.as_tensor(Xs[perm], device="cuda")
        dY = torch.as_tensor(Ys[perm], device="cuda")
        for s0 in range(0, ns - bs + 1, bs):
            t += 1
            want = log_every > 0 and (t % log_every == 0 or t == steps)
            loss = ctx.rbf_mlp_train_step(params, m, v, t, lr, dX[s0:s0 + bs], dY[s0:s0 + bs], bs, g,
                                          want_loss=want)
            if want:
                losses.append((t, loss))
            if t >= steps:
                break
    net = StopNet(torch, params.cpu().numpy(), fm, fs, om, os_, **rules)
    return net, losses


def predict(ctx, torch, net: StopNet, X):
    """Network outputs de-standardised: [B][2] = (ln l, t) for raw features X."""
    Xs = ((np.asarray(X, np.float64) - net.feat_mean.cpu().numpy()) / net.feat_std.cpu().numpy()).astype(np.float32)
    dX = torch.as_tensor(Xs, device="cuda")
    dY = torch.empty((Xs.shape[0], N_OUT), dtype=torch.float32, device="cuda")
    ctx.rbf_mlp_forward(net.params, dX, Xs.shape[0], dY)
    return dY.cpu().numpy().astype(np.float64) * net.out_std + net.out_mean


def solve(ctx, op, f, net: StopNet, state, coef):
    """Learned-stop HKT (rbf_learned_hkt); returns the LearnedInfo."""
    s = net.c_struct()
    return ctx.rbf_learned_hkt(op, f, s, state, coef)
