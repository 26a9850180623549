"""Host-side parts of the benchmark that run without a GPU: the record of the
host the CPU baseline ran on, and the oracle baseline scaled from a row-block
sample (used where the FP64 matrix is too large for the host oracle)."""
import os

import numpy as np

import bench
import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_host_info_fields():
    hi = bench.host_info()
    assert set(hi) == {"cores", "cpu", "blas"}
    assert isinstance(hi["cores"], int) and hi["cores"] >= 1
    assert isinstance(hi["cpu"], str) and hi["cpu"]
    assert isinstance(hi["blas"], str) and hi["blas"]


def test_scaled_oracle_baseline_on_a_small_casing():
    small = w.pump_like(300, 1200, seed=w.nodes.BASE_SEED + 652)
    assert small.n == 1500
    out = bench.cpu_baseline_rows(small, 0.1, 8.0, steps=20, rows=100, sample_steps=4)
    assert out["kind"] == "oracle" and out["unit"] == "HKT solutions/s"
    assert out["value"] > 0.0 and np.isfinite(out["value"])
    assert "100 of 1500 rows" in out["sample"] and "GCV-HKT(20)" in out["sample"]


def test_mf_pair_ops_f64_counts_every_pair_once():
    import bench
    for n, ni in [(1, 0), (1, 1), (7, 3), (12, 12), (9, 0)]:
        cost = {(True, True): 17, (False, False): 14}
        ref = sum(cost.get((i < ni, j < ni), 18) for i in range(n) for j in range(i + 1, n))
        ref += sum(16 if i < ni else 13 for i in range(n))
        assert bench.mf_pair_ops_f64(n, ni) == ref


def test_mf_pair_ops_counts_every_pair_once():
    import bench
    for n, ni in [(1, 0), (1, 1), (7, 3), (12, 12), (9, 0)]:
        cost = {(True, True): 12, (False, False): 9}
        ref = sum(cost.get((i < ni, j < ni), 13) for i in range(n) for j in range(i + 1, n))
        ref += sum(11 if i < ni else 8 for i in range(n))
        assert bench.mf_pair_ops(n, ni) == ref


def test_shipped_stopnet_file_matches_the_npz(tmp_path):
    """The binary stop-network file read by rbf_stopnet_load holds exactly the
    arrays of the shipped .npz, in the documented layout."""
    import numpy as np

    from paper_2511_09798_gb300 import learned
    pkg = os.path.join(ROOT, "paper_2511_09798_gb300")
    out = str(tmp_path / "w.bin")
    learned.write_stopnet_file(os.path.join(pkg, "stopnet_weights.npz"), out)
    raw = open(out, "rb").read()
    assert raw == open(os.path.join(pkg, "stopnet_weights.bin"), "rb").read()
    assert raw[:8] == b"RBFSTOP1"
    dims = np.frombuffer(raw[8:28], "<i4")
    assert list(dims) == [20, 128, 2, learned.N_PARAMS, 10]
    z = np.load(os.path.join(pkg, "stopnet_weights.npz"))
    off = 28
    for key, cnt in (("params", learned.N_PARAMS), ("feat_mean", 20), ("feat_std", 20), ("out_mean", 2),
                     ("out_std", 2)):
        assert np.array_equal(np.frombuffer(raw[off:off + 4 * cnt], "<f4"), z[key])
        off += 4 * cnt
    assert list(np.frombuffer(raw[off:off + 16], "<i4")) == [int(x) for x in z["rules"]]
    assert np.array_equal(np.frombuffer(raw[off + 16:off + 48], "<f8"), z["tols"])
    assert len(raw) == off + 48
