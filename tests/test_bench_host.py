"""bench.py's host arithmetic (no GPU): the algorithmic FP32 work per sample
rollout that every roofline figure divides by, and the job throughput."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import scenarios  # noqa: E402


def test_flops_per_sample_rollout_closed_forms():
    """T [n (9 d_u + f_dyn + 3 d_p + 4) + n(n-1)/2 (3 d_p + 1) + n m (3 d_p + 1)]."""
    uni = scenarios.WORKLOADS["unicycle_n8"]()             # d_u 2, d_p 2, f_dyn 31, no obstacles
    assert bench.flops_per_sample_rollout(uni) == 100 * (8 * (18 + 31 + 6 + 4) + 28 * 7)
    h3 = scenarios.WORKLOADS["holo3d_n16"]()               # d_u 3, d_p 3, f_dyn 24
    assert bench.flops_per_sample_rollout(h3) == 100 * (16 * (27 + 24 + 9 + 4) + 120 * 10)
    ob = scenarios.WORKLOADS["obstacles4_n16"]()           # d_u 2, d_p 2, f_dyn 16, 4 obstacles
    assert bench.flops_per_sample_rollout(ob) == 100 * (16 * (18 + 16 + 6 + 4) + 120 * 7 + 16 * 4 * 7)


def test_quoted_per_rollout_figures():
    """The per-rollout figures quoted in the design notes: 66.8 k, 222 k, 199 k."""
    f = {k: bench.flops_per_sample_rollout(scenarios.WORKLOADS[k]()) for k in
         ("unicycle_n8", "holo3d_n16", "obstacles4_n16")}
    assert round(f["unicycle_n8"] / 1e3, 1) == 66.8
    assert round(f["holo3d_n16"] / 1e3) == 222
    assert round(f["obstacles4_n16"] / 1e3) == 199


def test_fp32_peak_and_job_throughput():
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 80.54784) < 1e-9
    assert bench.job_throughput(1_024_000, 1, 16.0) == 1_024_000 / 0.016
    assert bench.job_throughput(1_024_000, 4, 20.0) == 4 * 1_024_000 / 0.020
