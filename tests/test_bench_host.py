"""Host-side logic of bench.py (no GPU): the DRAM-traffic entry is reported
only for the sweep source, workload and storage it was captured on; whole-job
values sum the replicas over the slowest rank's time; the bounded oracle
sample of the reference arm stays within its budget; the reference line of
the indexed lattice counts fluid nodes; the indexed lattice's host index
refuses bad input."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_sweep_traffic_only_for_the_captured_source_and_workload(monkeypatch):
    t = dict(bench.SWEEP_TRAFFIC)
    import hashlib

    src = os.path.join(ROOT, "paper_1005_2594_gb300", "csrc", "lb_sweep.cuh")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    monkeypatch.setattr(bench, "SWEEP_TRAFFIC", dict(t, sha=sha))
    assert bench.sweep_traffic(t["config"], t["store"]) == t["bytes"]
    assert bench.sweep_traffic("duct256", t["store"]) is None
    assert bench.sweep_traffic(t["config"], 1) is None
    monkeypatch.setattr(bench, "SWEEP_TRAFFIC", dict(t, sha="0" * 16))
    assert bench.sweep_traffic(t["config"], t["store"]) is None


def test_job_value_sums_replicas_over_the_slowest_rank():
    # 4 replicas of 2M sites, 100 steps, slowest rank 50 ms -> 4 * 2e8 / 0.05 / 1e6
    assert abs(bench.job_value(4, 2_000_000, 100, 50.0) - 16000.0) < 1e-9


def test_reference_sample_is_a_bounded_sub_box():
    from paper_1005_2594_gb300 import workloads

    p, X, q = workloads.shear_cell(n=128, phi=0.30, U=0.02, seed=1002)
    sp, sX, sq, desc = bench.reference_sample(p, X, q, 150.0, 20)
    assert sp["nz"] == p["nz"] and sp["nx"] <= p["nx"] and sp["ny"] <= p["ny"]
    frac = sp["nx"] * sp["ny"] / (p["nx"] * p["ny"])
    # the cost model of the sample (12 s per 128^3 step with 1022 cells) fits the budget
    assert 12.0 * frac * frac * 20 <= 150.0 or (sp["nx"], sp["ny"]) == (16, 16)
    assert abs(len(sX) - len(X) * frac) <= 1


def test_oracle_on_all_cores_aggregates_processes():
    """the all-core CPU baseline: spawned processes, each stepping its own
    copy, their site updates summed over the slowest one's time"""
    from paper_1005_2594_gb300 import workloads

    p, X, q = workloads.small_shear()
    v, n, t = bench.oracle_all_cores(p, X, q, None, 0, 1, procs=2)
    assert n == 2 and t > 0
    assert abs(v - 2 * 32 ** 3 / t / 1e6) < 1e-9
    assert 1 <= bench.host_cores(32 ** 3) <= (os.cpu_count() or 1)


def test_sweep_kernel_label_follows_the_default_variant():
    # with cells one node per thread; without, the bulk-copy pipeline where rows allow it
    assert bench.sweep_kernel(128, 0).startswith("k_lb_step ") and "FP32" in bench.sweep_kernel(128, 0)
    assert "k_lb_step_bulk" in bench.sweep_kernel(128, 0, cells=False)
    assert "k_lb_step_bulk" in bench.sweep_kernel(256, 1, cells=False) and "BF16" in bench.sweep_kernel(256, 1, cells=False)
    assert "k_lb_step_pipe" in bench.sweep_kernel(30, 0, cells=False)
    assert bench.sweep_kernel(36, 2, cells=False).startswith("k_lb_step ") and "FP16" in bench.sweep_kernel(36, 2)
    # an explicit variant: its kernel where the rows and the storage allow it
    assert bench.sweep_kernel(128, 0, 5).startswith("k_lb_step_rows ")
    assert "4 planes" in bench.sweep_kernel(128, 1, 4)
    assert bench.sweep_kernel(36, 2, 5).startswith("k_lb_step ")
    assert bench.sweep_kernel(64, 1, 2).startswith("k_lb_step ")


def test_clock_sampler_reports_without_a_gpu():
    c = bench.ClockSampler(0)
    c.start()
    out = c.stop()
    assert "samples" in out and "reasons" in out


def test_reference_arm_line_for_the_vessel_loop_counts_fluid_nodes():
    """--impl reference on the indexed-lattice config: the oracle's rate in
    fluid-node updates, the unit saying so, as the GPU line does"""
    import argparse

    args = argparse.Namespace(config="vessel_loop", steps=1, warmup=0)
    out = bench.run_reference(args, 1, 0)
    assert out["impl"] == "reference" and out["unit"].endswith("(fluid nodes)")
    assert out["cpu_baseline"]["unit"] == out["unit"] == out["e2e"]["unit"]
    assert out["value"] > 0 and out["cpu_baseline"]["cores"] >= 1
    assert "256x128x32" in out["config"]["sample"]


def test_sparse_index_rejects_bad_input():
    import ctypes

    import numpy as np
    import pytest

    from paper_1005_2594_gb300 import bloodlb as bl
    from paper_1005_2594_gb300 import workloads

    p = workloads.base_params(6, 5, 4, periodic=(1, 0, 1))
    with pytest.raises(ValueError):
        bl.bl_sparse_index_build(p, np.zeros(7, dtype=np.uint8))  # wrong size
    with pytest.raises(bl.BloodLBError):
        bl.bl_sparse_index_build(p, np.full(6 * 5 * 4, 9, dtype=np.uint8))  # no wall id 8
    q = workloads.base_params(6, 2, 4, periodic=(1, 0, 1))  # a walled axis needs fluid between its walls
    n = ctypes.c_int64(0)
    assert bl.lib().bl_sparse_index_build(ctypes.byref(bl.lb_params(q)), None, ctypes.byref(n), None, None) \
        == bl.BL_EINVAL
