"""The eigensolve driver (Algorithm 1 over the C ABI, phases timed) on the 4^3-cell workload:
every run converges, and the mixed-precision runs reach the FP64 run's Ritz values within
1e-7 Ha."""
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_driver_runs_converge_and_agree():
    from paper_2605_30128_gb300.eigensolve import run
    w = workloads.workload("cfg1")
    out = run(w, ["chfsi_fp64", "rchfsi_fp32_df", "rchfsi_fp32"], cycles=200, tol=1e-9, nwanted=28)
    runs = out["runs"]
    assert set(runs) == {"chfsi_fp64", "rchfsi_fp32_df", "rchfsi_fp32"}
    for name, rec in runs.items():
        assert rec["final_max_residual"] < 1e-9, (name, rec["history"][-3:])
        assert 0 < rec["cycles"] < 200
        assert abs(sum(rec["split"].values()) - 1.0) < 1e-12
    for name in ("rchfsi_fp32_df", "rchfsi_fp32"):
        assert runs[name]["max_ritz_diff_vs_chfsi_fp64"] < 1e-7
