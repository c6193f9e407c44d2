"""Host logic of bench.py on CPU: the oracle-based CPU baseline and reference
arm (bounded samples scaled by the counts of the oracle's own full solve)."""
import json

import numpy as np

import bench
import sw_inputs as si


def test_counts_script_uses_the_bench_inputs():
    """oracle/solve_counts.py draws its null-vector guesses with
    sw_inputs.null_vector_guesses; they must be the bench's."""
    _, psi0 = bench.gauge_and_psi0(32, bench.WORKLOAD["beta"], 1, "cpu")
    ref = si.null_vector_guesses(32, 32, bench.WORKLOAD["nvec"], 3,
                                 [tuple(b) for b in bench.WORKLOAD["blocks"]])
    assert len(psi0) == len(ref) and all(np.array_equal(a, b) for a, b in zip(psi0, ref))


def test_stored_counts_describe_the_workload():
    rec = bench.oracle_counts(bench.WORKLOAD["L"])
    assert rec is not None
    w = rec["workload"]
    assert (w["L"], w["mass"], w["nvec"], w["tol"]) == (
        bench.WORKLOAD["L"], bench.WORKLOAD["mass"], bench.WORKLOAD["nvec"], bench.WORKLOAD["tol"])
    assert [list(b) for b in w["blocks"]] == bench.WORKLOAD["blocks"]
    assert w["coarsest_maxiter"] == bench.WORKLOAD["coarsest_maxiter"]
    assert rec["stats"]["converged"] and rec["stats"]["true_resid"] <= 1e-10
    c = rec["counts"]
    assert c["S"] == rec["stats"]["fine_applies"]
    # every coarsest CGNE iteration applies A_hat and its adjoint once
    assert c["A3"] >= 2 * rec["stats"]["coarsest_iters"]
    # wall time over the time of the counted applications alone (near 1 up to timing noise:
    # the coarsest applications dominate the oracle's solve)
    assert 0.8 <= rec["overhead_ratio"] <= 2.0
    assert bench.oracle_counts(bench.WORKLOAD["L"] // 2) is None


def test_reference_arm_bounded_sample(tmp_path, monkeypatch, capsys):
    rec = {"workload": {"L": 32}, "counts": {"S": 10, "A2": 20, "A3": 30},
           "overhead_ratio": 1.5, "machine": {"processor": "test"}}
    path = tmp_path / "counts.json"
    path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "COUNTS_FILE", str(path))

    class Args:
        L, sweeps, warmup, steps = 32, 2, 1, 2

    bench.run_reference(Args, 0, 1)
    line = json.loads(capsys.readouterr().out)
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["cpu_baseline"]["cores"] == 1
    assert abs(line["ms_per_step"] * 1e-3 * line["value"] - 1.0) < 1e-9
    assert line["e2e"]["h2d_bytes_per_step"] == 0

    class Other(Args):
        L = 64

    bench.run_reference(Other, 0, 1)
    assert "unavailable" in json.loads(capsys.readouterr().out)


def test_profiled_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from a committed ncu summary only while
    the kernel source still has the SHA-1 the summary records: the current
    profile matches the current source, and a changed source (or a missing
    key) gives None instead of a stale figure."""
    import hashlib
    import os
    v = bench._profiled_traffic("k_cgne64_fp64_256.md", "paper_1801_07823_gb300/csrc/cgne64.cu",
                                "dram_bytes_per_iteration")
    assert v is not None and v > 0
    (tmp_path / "profiles").mkdir()
    (tmp_path / "src.cu").write_text("kernel v1\n")
    sha = hashlib.sha1(b"kernel v1\n").hexdigest()
    (tmp_path / "profiles" / "p.md").write_text(
        f"dram_bytes_per_iteration: 1234\nsource_sha1 (src.cu): {sha}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._profiled_traffic("p.md", "src.cu", "dram_bytes_per_iteration") == 1234.0
    assert bench._profiled_traffic("p.md", "src.cu", "other_key") is None
    (tmp_path / "src.cu").write_text("kernel v2\n")
    assert bench._profiled_traffic("p.md", "src.cu", "dram_bytes_per_iteration") is None
    assert os.path.exists(tmp_path / "profiles" / "p.md")
