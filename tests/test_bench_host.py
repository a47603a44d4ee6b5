"""Host logic of bench.py: counting eigenpairs and the per-result error report."""
import numpy as np


def test_count_good_and_accuracy_summary():
    import bench
    gold = np.array([1.0 + 1.0j, 1.1 + 1.0j, 0.9 + 1.05j])
    lam = np.array([1.0 + 1.0j + 1e-12, 1.1 + 1.0j + 5e-10, 0.9 + 1.05j, 3.0 + 0j])
    rr = np.array([1e-12, 1e-12, 2e-10, 1e-14])
    acc = bench.new_accuracy()
    # inside the circle |l - (1+1j)| < 0.5: the first three; the first is good, the
    # second misses the eigenvalue bar, the third the residual bar
    assert bench.count_good(lam, rr, gold, 1.0 + 1.0j, 0.5, 0.5, acc=acc) == 1
    s = bench.accuracy_summary(acc)
    assert s["pairs"] == 3
    assert np.isclose(s["max_rel_eig_err"], 5e-10 / abs(gold[1]), rtol=1e-3)
    assert s["max_relres"] == 2e-10
    assert bench.accuracy_summary(bench.new_accuracy()) == {"pairs": 0}


def test_configs_are_consistent_with_generators_and_stored_contours():
    import json
    import os
    import bench
    import workloads
    gold = json.load(open(os.path.join(bench.ROOT, "tests", "golden", "contours.json")))
    assert "qep_mixed_n4096" in bench.WORKLOADS
    for name, spec in bench.WORKLOADS.items():
        assert callable(getattr(workloads, spec["gen"])), name
        assert spec["precision"] in bench.DTYPES, name
        assert 0 < spec["tol"] <= 1e-10 and spec["maxit"] >= 10, name
        c = gold[name]
        if spec.get("mixed"):
            assert "problems" in c
        elif spec.get("slices"):
            assert len(c["centers"]) == len(c["eigs_inside"])
        else:
            assert len(c["eigs_inside"]) == c["count"]
            assert c["generator"].startswith(spec["gen"] + "(n=%d" % spec["n"])


def test_phase_work_counts_the_stated_flops():
    import bench
    spec = dict(bench.WORKLOADS["qep_mixed_n4096"])
    c = {"m0": 96, "nc": 16}
    n, m0 = 4096, 96
    assert bench.phase_work("lu", spec, c, 6, 3) == 16 * (8.0 / 3.0) * n ** 3      # 2.93e12
    assert bench.phase_work("solve", spec, c, 6, 3) == 5 * 16 * 8.0 * n * n * m0    # none after the last
    pairs = bench.DIGIT_SLICES * (bench.DIGIT_SLICES + 1) // 2
    a3 = bench.phase_work("apply", spec, c, 6, 3)
    assert a3 == 6 * 3 * pairs * 2.0 * n * (2 * n) * (2 * m0)
    # a diagonal term is scaled, not sliced: only the sliced terms count
    assert bench.phase_work("apply", spec, c, 6, 3, nterms_sliced=2) == a3 * 2 / 3
    spec["precision"] = "fp32"
    assert bench.phase_work("apply", spec, c, 6, 3) == 6 * 3 * 8.0 * n * n * m0
    assert bench.phase_work("reduced", spec, c, 6, 3) == 6 * (40.0 / 3.0 + 10.0) * (2 * m0) ** 3


def test_phase_peaks_follow_the_arithmetic_of_each_phase():
    import bench
    pk = {"tf32_tflops": 1044.0, "fp32_simt_tflops": 69.9, "fp64_tflops": 1.10,
          "bf16_tflops": 1911.8, "bf16_tflops_sustained": 1726.1, "source": "measured"}
    assert bench.phase_peak("lu", "fp32_i8", pk, 2070.0)[:2] == (1044.0 / 3.0, "tensor")
    assert bench.phase_peak("apply", "fp32_i8", pk, 2070.0)[:2] == (1726.1, "tensor")
    assert bench.phase_peak("reduced", "fp32_i8", pk, 2070.0)[:2] == (69.9, "alu")
    assert bench.phase_peak("lu", "fp64", pk, 2070.0)[:2] == (1.10, "alu")
    # without live probes: TF32 = half the BF16 figure, FP32 lanes nominal at the clock
    pk0 = {"bf16_tflops": 1911.8, "bf16_tflops_sustained": 1726.1, "source": "measured"}
    assert bench.phase_peak("solve", "fp32", pk0, 2070.0)[0] == 1911.8 * 0.5 / 3.0
    assert abs(bench.phase_peak("reduced", "fp32", pk0, 1035.0)[0]
               - bench.FP32_SIMT_TFLOPS_AT_MAX / 2) < 1e-9


def test_match_count_takes_each_reference_eigenvalue_once():
    import bench
    ref = np.array([1.0 + 1.0j, 2.0 + 0.0j])
    lam = np.array([1.0 + 1.0j, 1.0 + 1.0j + 1e-14, 2.0 + 1e-9j, 2.0 + 0.0j])
    rr = np.array([1e-12, 1e-12, 1e-12, 1e-9])
    # the second copy of 1+1i finds its reference taken; 2+1e-9i misses by 5e-10
    # relative; the last misses the residual bar
    assert bench.match_count(lam, rr, ref) == 1
    assert bench.match_count(lam, rr, np.array([])) == 0


def test_reference_arm_prints_one_complete_json_line(capsys):
    """`bench.py --impl reference` on the n = 256 QEP (one FP64 oracle solve):
    one JSON line with the contract's keys, all 16 pairs counted."""
    import argparse
    import json
    import bench
    bench.run_reference(argparse.Namespace(workload="qep_plain_n256", seed=0, warmup=0, steps=1))
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and abs(d["value"] - 16 / (d["ms_per_step"] / 1e3)) < 1e-6 * d["value"]
    assert d["config"]["workload"] == "qep_plain_n256"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
