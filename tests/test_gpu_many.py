"""GPU: several independent GKB runs and projected solves spread over the
context's lanes (rbf_gkb_many, rbf_hkt_many).  They run the same kernels as
rbf_gkb / rbf_hkt on other streams, so every result must equal the
single-run call bitwise, whatever the lane count, for assembled FP64, mixed
and matrix-free operators, with and without assembly by the lanes, and with a
run that breaks down early."""
import numpy as np
import pytest

import workloads as w
from oracle import gkb as OG
from oracle import mq as OM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_09798_gb300 import rbfkr
    return rbfkr


def _cases(R):
    rng = np.random.Generator(np.random.PCG64(61))
    base = rng.uniform(0, 1, (12, 3))
    dup = w.NodeSet(np.concatenate([base, base]), 14, "cube", "dup24")  # repeated centres: rank <= 12, breakdown
    sets = [w.cube_faces_random(900, 0.3, rng), w.sphere_fibonacci_ball(200, 700, seed=9), dup,
            w.cube_faces_random(1300, 0.3, rng), w.cube_faces_random(500, 0.4, rng)]
    kinds = [(R.RBF_ASSEMBLED, R.RBF_FP64), (R.RBF_MATRIX_FREE, R.RBF_MIXED), (R.RBF_ASSEMBLED, R.RBF_FP64),
             (R.RBF_ASSEMBLED, R.RBF_MIXED), (R.RBF_MATRIX_FREE, R.RBF_FP64)]
    cs, ks = [0.3, 0.2, 0.3, 0.25, 0.35], [2.0, 4.0, 2.0, 3.0, 1.5]
    return sets, kinds, cs, ks


def _ops(ctx, R, sets, kinds, cs, ks, fill_nan=False):
    ops, keep = [], []
    for ns, (storage, prec), c, k in zip(sets, kinds, cs, ks):
        nodes = torch.as_tensor(ns.soa(), device="cuda")
        A, lda = None, 0
        if storage == R.RBF_ASSEMBLED:
            lda = R.padded_lda(ns.n, prec)
            dt = torch.float64 if prec == R.RBF_FP64 else torch.float32
            A = torch.full((ns.n, lda), float("nan"), dtype=dt, device="cuda")
        op = ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, c, k, storage, prec, R.RBF_FORM_C, A, lda)
        if A is not None and not fill_nan:
            ctx.rbf_assemble(op)
        ops.append(op)
        keep.append((nodes, A))
    return ops, keep


@pytest.mark.parametrize("lanes", [1, 2, 3])
@pytest.mark.parametrize("assemble", [False, True])
def test_gkb_many_equals_single_runs(R, lanes, assemble):
    sets, kinds, cs, ks = _cases(R)
    steps = 24
    ctx = R.Context(0)
    fs = [torch.as_tensor(w.plane_wave_rhs(s, k), device="cuda") for s, k in zip(sets, ks)]
    ops1, keep1 = _ops(ctx, R, sets, kinds, cs, ks)
    ref = []
    for op, f, ns in zip(ops1, fs, sets):
        st, W, Z, al, be = R.make_state(torch, ns.n, steps)
        ctx.rbf_gkb(op, f, steps, st)
        ref.append((st.steps_done, st.breakdown, st.c_hat, W.clone(), Z.clone(), al.clone(), be.clone()))
    ops2, keep2 = _ops(ctx, R, sets, kinds, cs, ks, fill_nan=assemble)
    states, bufs = [], []
    for ns in sets:
        st, *b = R.make_state(torch, ns.n, steps)
        states.append(st)
        bufs.append(b)
    ctx.rbf_gkb_many(ops2, fs, steps, states, lanes=lanes, assemble=assemble)
    for i, ns in enumerate(sets):
        sd, bd, ch, W, Z, al, be = ref[i]
        assert (states[i].steps_done, states[i].breakdown) == (sd, bd), i
        assert states[i].c_hat == ch, i
        W2, Z2, al2, be2 = bufs[i]
        l = sd
        assert torch.equal(al2[:l], al[:l]) and torch.equal(be2[:l + 1], be[:l + 1]), i
        assert torch.equal(Z2[:l], Z[:l]) and torch.equal(W2[:l + 1], W[:l + 1]), i
        if assemble and keep1[i][1] is not None:
            assert torch.equal(keep2[i][1][:, :ns.n], keep1[i][1][:, :ns.n]), i
    # the repeated-node run broke down like the oracle's
    g = OG.gkb(OM.assemble(sets[2].X, sets[2].n_interior, cs[2], ks[2]), None, w.plane_wave_rhs(sets[2], ks[2]),
               steps)
    assert g.steps_done < steps and states[2].steps_done == g.steps_done
    # projected solves of all runs at once equal the single calls
    coefs = [torch.empty(ns.n, dtype=torch.float64, device="cuda") for ns in sets]
    infos = ctx.rbf_hkt_many(states, R.RBF_GCV, 0.0, coefs, lanes=lanes)
    for i, ns in enumerate(sets):
        c1 = torch.empty(ns.n, dtype=torch.float64, device="cuda")
        inf1 = ctx.rbf_hkt(states[i], R.RBF_GCV, 0.0, c1)
        assert torch.equal(c1, coefs[i]), i
        assert infos[i].lambda_ == inf1.lambda_ and infos[i].index == inf1.index, i
    ctx.close()


def test_many_pair_assembly_of_operators_sharing_nodes(R):
    """FP64 operators on one node array with one c and form, differing in k, are
    assembled two at a time by rbf_gkb_many: every matrix equals its own
    rbf_assemble bitwise (both forms, an odd operator left over, a mixed one
    not paired), and so do the GKB runs."""
    ns = w.cube_faces_random(700, 0.3, np.random.Generator(np.random.PCG64(91)))
    nodes = torch.as_tensor(ns.soa(), device="cuda")
    specs = [(R.RBF_FP64, R.RBF_FORM_C, 2.0), (R.RBF_MIXED, R.RBF_FORM_C, 3.0), (R.RBF_FP64, R.RBF_FORM_C, 5.0),
             (R.RBF_FP64, R.RBF_FORM_EPS, 2.0), (R.RBF_FP64, R.RBF_FORM_C, 3.5), (R.RBF_FP64, R.RBF_FORM_EPS, 4.0)]
    steps = 12
    ctx = R.Context(0)

    def make(fill):
        ops, mats = [], []
        for prec, form, k in specs:
            lda = R.padded_lda(ns.n, prec)
            dt = torch.float64 if prec == R.RBF_FP64 else torch.float32
            A = torch.full((ns.n, lda), float("nan"), dtype=dt, device="cuda")
            op = ctx.rbf_operator_init(nodes, ns.n, ns.n_interior, 0.3, k, R.RBF_ASSEMBLED, prec, form, A, lda)
            if fill:
                ctx.rbf_assemble(op)
            ops.append(op)
            mats.append(A)
        return ops, mats
    ops1, mats1 = make(True)
    ops2, mats2 = make(False)
    fs = [torch.as_tensor(w.plane_wave_rhs(ns, k), device="cuda") for _, _, k in specs]
    ref = []
    for op, f in zip(ops1, fs):
        st, W, Z, al, be = R.make_state(torch, ns.n, steps)
        ctx.rbf_gkb(op, f, steps, st)
        ref.append((W, al))
    states, bufs = [], []
    for _ in specs:
        st, *b = R.make_state(torch, ns.n, steps)
        states.append(st)
        bufs.append(b)
    ctx.rbf_gkb_many(ops2, fs, steps, states, lanes=2, assemble=True)
    torch.cuda.synchronize()
    for i in range(len(specs)):
        assert torch.equal(mats2[i][:, :ns.n], mats1[i][:, :ns.n]), i
        assert torch.equal(bufs[i][0], ref[i][0]) and torch.equal(bufs[i][2], ref[i][1]), i
    ctx.close()


def test_many_busy_time_and_counts(R):
    """Product timing with lanes: the union of the launch intervals never exceeds
    their sum, and every product launch is counted."""
    sets, kinds, cs, ks = _cases(R)
    steps = 10
    ctx = R.Context(0, timing=2)
    ops, keep = _ops(ctx, R, sets, kinds, cs, ks)
    fs = [torch.as_tensor(w.plane_wave_rhs(s, k), device="cuda") for s, k in zip(sets, ks)]
    states = [R.make_state(torch, ns.n, steps)[0] for ns in sets]
    ctx.rbf_get_counters(reset=True)
    ctx.rbf_gkb_many(ops, fs, steps, states, lanes=2)
    cnt = ctx.rbf_get_counters(reset=True)
    assert cnt["product_launches"][0] == cnt["product_launches"][1] == steps * len(sets)
    assert 0 < cnt["product_busy_ms"] <= sum(cnt["product_ms"]) * (1 + 1e-6)
    assert cnt["launches"] >= 4 * steps * len(sets)
    ctx.close()


def test_many_rejects_bad_arguments(R):
    ctx = R.Context(0)
    ns = w.cube_faces_random(300, 0.3, np.random.Generator(np.random.PCG64(3)))
    (op,), keep = _ops(ctx, R, [ns], [(R.RBF_MATRIX_FREE, R.RBF_MIXED)], [0.3], [2.0])
    f = torch.as_tensor(w.plane_wave_rhs(ns, 2.0), device="cuda")
    st = R.make_state(torch, ns.n, 5)[0]
    with pytest.raises(R.RbfError) as e:
        ctx.rbf_gkb_many([op], [f], 6, [st])  # steps above the capacity
    assert e.value.status == R.RBF_ERR_INVALID
    with pytest.raises(R.RbfError) as e:
        ctx.rbf_gkb_many([op], [f], 5, [st], lanes=9)
    assert e.value.status == R.RBF_ERR_INVALID
    ctx.close()


def test_many_more_runs_than_lanes_and_stream_order(R):
    """Ten runs with the default lane count (capped at 8, and by the half-step
    kernel's co-residency), inputs written on the context stream just before
    the call (the lanes start after that work), results equal to single runs."""
    rng = np.random.Generator(np.random.PCG64(81))
    sets = [w.cube_faces_random(int(n), 0.3, rng) for n in rng.integers(300, 1400, 10)]
    steps = 15
    stream = torch.cuda.Stream()
    ctx = R.Context(0, stream=stream)
    ops, keep = _ops(ctx, R, sets, [(R.RBF_ASSEMBLED, R.RBF_FP64)] * 10, [0.3] * 10, [2.0] * 10)
    torch.cuda.synchronize()
    host = [torch.as_tensor(w.plane_wave_rhs(s, 2.0)).pin_memory() for s in sets]
    fs = [torch.zeros(s.n, dtype=torch.float64, device="cuda") for s in sets]
    states = [R.make_state(torch, s.n, steps)[0] for s in sets]
    with torch.cuda.stream(stream):
        for f, h in zip(fs, host):
            f.copy_(h, non_blocking=True)  # enqueued on the context stream
        ctx.rbf_gkb_many(ops, fs, steps, states)
    for i, s in enumerate(sets):
        st1, W1, Z1, a1, b1 = R.make_state(torch, s.n, steps)
        ctx.rbf_gkb(ops[i], fs[i], steps, st1)
        torch.cuda.synchronize()
        assert st1.steps_done == states[i].steps_done == steps
        assert torch.equal(a1, states[i]._keep[2]) and torch.equal(W1, states[i]._keep[0]), i
    ctx.close()
