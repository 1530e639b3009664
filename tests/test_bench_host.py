"""Host-side logic of bench.py (no GPU): the DRAM-traffic entry is reported
only for the sweep source, workload and storage it was captured on; whole-job
values sum the replicas over the slowest rank's time; the bounded oracle
sample of the reference arm stays within its budget."""
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
