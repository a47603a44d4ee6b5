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
