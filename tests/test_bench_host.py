"""Host-side parts of the benchmark that run without a GPU: the record of the
host the CPU baseline ran on, and the oracle baseline scaled from a row-block
sample (used where the FP64 matrix is too large for the host oracle)."""
import numpy as np

import bench
import workloads as w


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


def test_mf_ops_per_entry_mix():
    # 11 FP32-pipe operations per PDE entry, 8 per Dirichlet entry, averaged over the rows
    assert bench.mf_ops_per_entry(10, 10) == 11
    assert bench.mf_ops_per_entry(10, 0) == 8
    assert bench.mf_ops_per_entry(4, 1) == (11 + 3 * 8) / 4
