"""The GPU arm's CPU-baseline leg, without a GPU: the oracle's full hot-path step run in a spawned
process pinned to one host core (as run_ours starts it before its first GPU call) returns its measured
parts, the oracle's own iteration count and true residual, and the arrays the error comparison reads
(on the small 4x4x4x8 workload)."""

import numpy as np

import bench


def test_oracle_job_in_a_spawned_process():
    jobs = bench.OracleJobs([("t_4x4x4x8", True)])
    try:
        r = jobs.result("t_4x4x4x8", timeout=300)
        assert "error" not in r, r
        assert r["cg_iters"] > 0 and r["mdagm_applications"] >= r["cg_iters"]
        assert r["true_rel_resid"] <= 1e-8
        assert abs(r["step_s"] - (r["clover_s"] + r["solve_s"] + r["force_s"])) < 1e-12
        x, F, Mb = (jobs.array("t_4x4x4x8", k) for k in ("x", "F", "Mb"))
        assert x.shape == (4 * 4 * 4 * 8 // 2, 4, 3) and Mb.shape == x.shape
        assert F.shape == (8, 4, 4, 4, 4, 3, 3)
        # the force is traceless anti-Hermitian
        assert np.max(np.abs(F + np.conj(np.swapaxes(F, -1, -2)))) < 1e-12
    finally:
        jobs.close()


def test_step_unit_names_the_lattice():
    assert bench.step_unit(bench.workload_params("c1_16^4")) == "ms per hot-path step (16^4, solve to 1e-8)"
    assert bench.step_unit(bench.workload_params("t_4x4x4x8")) == "ms per hot-path step (4x4x4x8, solve to 1e-8)"
