"""Shape and structure of the seeded synthetic workloads."""
import numpy as np

import workloads as w
from workloads.nodes import inside


def test_cube_grid_counts():
    ns = w.cube_grid(10)
    assert (ns.n, ns.n_interior, ns.n_boundary) == (1000, 512, 488)
    XI, XB = ns.X[:512], ns.X[512:]
    assert np.all((XI > 0) & (XI < 1))
    assert np.all(np.any((XB == 0) | (XB == 1), axis=1))


def test_cube_halton_counts_and_unique_boundary():
    ns = w.cube_faces_halton(8000, 21)
    assert ns.n_boundary == 21 ** 3 - 19 ** 3 == 2402
    assert ns.n_interior == 5598
    B = ns.X[ns.n_interior:]
    assert np.unique(B, axis=0).shape[0] == B.shape[0]
    assert np.all((ns.X[:ns.n_interior] > 0) & (ns.X[:ns.n_interior] < 1))
    assert np.array_equal(ns.X, w.cube_faces_halton(8000, 21).X)  # seeded


def test_scrambled_halton_is_low_discrepancy():
    P = w.scrambled_halton(4096, np.random.Generator(np.random.PCG64(1)))
    # every 1/8-cube cell receives close to its share (Halton fills evenly)
    cells = np.floor(P * 2).astype(int)
    counts = np.bincount(cells[:, 0] * 4 + cells[:, 1] * 2 + cells[:, 2], minlength=8)
    assert np.all(np.abs(counts - 512) <= 8)


def test_sphere_set():
    ns = w.sphere_fibonacci_ball(400, 1600, seed=11)
    assert np.allclose(np.linalg.norm(ns.X[1600:], axis=1), 1.0)
    assert np.all(np.linalg.norm(ns.X[:1600], axis=1) < 1.0)


def test_batch_instances_ranges():
    inst = w.batch_instances(12)
    for ns in inst:
        p = ns.params
        assert 2000 <= ns.n <= 16000
        assert 0.05 <= p["c"] <= 1.0 and 1.0 <= p["k"] <= 20.0
        assert abs(np.linalg.norm(p["d"]) - 1) < 1e-12
        share = ns.n_boundary / ns.n
        assert (0.25 < share < 0.36) if ns.domain == "cube" else abs(share - 0.2) < 1e-3


def test_pump_like_small():
    ns = w.pump_like(300, 1200, seed=5)
    assert ns.n == 1500
    assert np.all(inside("pump", ns.X[:1200]))
    P = w.test_points(ns, 200)
    assert np.all(inside("pump", P))


def test_paper_shaped_node_sets():
    import numpy as np
    import workloads as w
    for dom in ("cube", "sphere"):
        for dist in ("random", "uniform", "halton"):
            for n in (359, 2154):
                ns = w.paper_nodes(dom, dist, n, 9798 + 7)
                assert abs(ns.n - n) <= 0.06 * n, (dom, dist, n, ns.n)
                X = ns.X
                I, B = X[: ns.n_interior], X[ns.n_interior:]
                if dom == "cube":
                    assert np.all((I > 0) & (I < 1))
                    assert np.all(np.any((B == 0) | (B == 1), axis=1))
                else:
                    assert np.all(np.sum(I * I, axis=1) < 1)
                    assert np.allclose(np.sum(B * B, axis=1), 1.0)
                assert len(np.unique(X.round(12), axis=0)) == ns.n
    # seeded: the same seed gives the same set
    a = w.paper_nodes("cube", "halton", 359, 5)
    b = w.paper_nodes("cube", "halton", 359, 5)
    assert np.array_equal(a.X, b.X)


def test_stop_instances_casing_share(monkeypatch):
    """pump_share = 0 keeps the cube/sphere draws; a positive share mixes in
    casing-like node sets drawn without repetition from the pool."""
    import workloads.nodes as N
    small = w.pump_like(400, 1600, seed=N.BASE_SEED + 651)
    monkeypatch.setattr(N, "_PUMP_POOL", (small.X[small.n_interior:].copy(), small.X[:small.n_interior].copy()))
    plain = w.stop_instances(12, 300, 600)
    again = w.stop_instances(12, 300, 600, pump_share=0.0)
    assert {s.domain for s in plain} <= {"cube", "sphere"}
    for a, b in zip(plain, again):
        assert a.domain == b.domain and np.array_equal(a.X, b.X) and a.params["c"] == b.params["c"]
    mixed = w.stop_instances(24, 300, 600, pump_share=0.5)
    pumps = [s for s in mixed if s.domain == "pump"]
    assert pumps
    for s in pumps:
        assert s.n_boundary == round(0.2 * s.n)
        assert np.unique(s.X, axis=0).shape[0] == s.n
        assert inside("pump", s.X[:s.n_interior]).all()
        assert s.params["rhs"] in ("plane", "gauss")
        if s.params["rhs"] == "gauss":
            assert inside("pump", s.params["center"][None, :]).all()
