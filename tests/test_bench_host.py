"""Host-side pieces of bench.py (CPU): the all-core oracle baseline's worker pool and the
memory-side fractions reported beside the transport's ALU roofline."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_oracle_pool_runs_even_samples_of_every_spot():
    import bench
    from paper_1409_8336_gb300 import workloads as W

    p = W.water_box((8, 8, 16), 0.2, [W.spot_row(70.0), W.spot_row(110.0)], n_batches=2)
    pool = bench.OraclePool(p, 2000, procs=2)
    try:
        assert list(pool.cnt) == [1000, 1000] and list(pool.first) == [0, 1000]
        rate, done, dt = pool.rate(0.05, rate1=2000.0)
        # per = max(procs, rate1 x seconds x procs / spots) = 100 histories of each spot
        assert done == 200 and dt > 0 and rate == pytest.approx(done / dt)
    finally:
        pool.close()


def test_memory_fractions():
    import bench

    pk = {"hbm_gbs": 5000.0}
    m = bench.memory_fractions(pk, steps_per_step=1e8, span_ms=2.0, traffic=4e7, launches_per_step=1.0)
    assert m["algorithmic_gbs"] == pytest.approx(21 * 1e8 / 2e-3 / 1e9)
    assert m["algorithmic_frac"] == pytest.approx(m["algorithmic_gbs"] / 5000.0)
    assert m["dram_gbs"] == pytest.approx(4e7 / 2e-3 / 1e9) and m["dram_frac"] == pytest.approx(0.004)
    assert bench.memory_fractions(pk, 1e8, 2.0, None, 1.0)["dram_frac"] is None


def test_profiler_figures_are_null_for_other_sources(monkeypatch):
    import bench

    monkeypatch.setitem(bench.TRAFFIC, "bytes_per_history", 50.0)
    if bench._sources_match():
        assert bench.traffic_per_launch(1e6) == pytest.approx(5e7)
        assert bench.ncu_fractions()["simt_efficiency"] == pytest.approx(bench.NCU["threads_per_instruction"] / 32)
    monkeypatch.setattr(bench, "KERNEL_SHA256", "0" * 64)
    assert bench.traffic_per_launch(1e6) is None
    assert bench.ncu_fractions() is None
    monkeypatch.setitem(bench.TRAFFIC, "bytes_per_history", None)
    assert bench.traffic_per_launch(1e6) is None
