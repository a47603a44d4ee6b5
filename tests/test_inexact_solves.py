"""Algorithm 1 with inexact node solves (CPU only).

Sec. 4.2 reads the filter as residual inverse iteration: Step 4 solves with the
block residual T(X, Lambda) on the right, so a node solve's relative error
multiplies a quantity that vanishes at convergence.  With Steps 1-3 in FP64,
node solves in FP32 or emulated TF32 must therefore reach the same tolerance in
about the same number of iterations, and the eigenvalues must agree with the
FP64 run's to rounding of the FP64 steps -- far below the solves' own error
(6e-8 for FP32, 5e-4 for TF32).  A Step 4 that solved against X rather than
against the residual would leave the eigenvalues at the solve's precision.
"""
import json
import os

import numpy as np
import pytest

import oracle.nlfeast_ref as O
from tests import precision_study as S
from workloads import config1_qep, start_block


@pytest.fixture(autouse=True)
def _few_blas_threads():
    """The products here are small (n = 256, m0 = 24): many BLAS threads only
    contend.  threadpoolctl is optional."""
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:
        yield
        return
    with threadpool_limits(limits=2, user_api="blas"):
        yield


def test_tf32_rounding_is_round_to_nearest_even():
    x = np.array([1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 1 + 2.0 ** -10 + 2.0 ** -12,
                  -1 - 2.0 ** -11 - 2.0 ** -20, 3.0, 0.0], dtype=np.float32)
    want = np.array([1, 1 + 2.0 ** -9, 1 + 2.0 ** -10, -1 - 2.0 ** -10, 3, 0], dtype=np.float32)
    assert np.array_equal(S.tf32(x), want)


@pytest.mark.parametrize("mode,eps", [("fp32", 2.0 ** -24), ("tf32x3", 2.0 ** -24),
                                      ("tf32", 2.0 ** -11)])
def test_emulated_blocked_lu_solves(mode, eps):
    """The emulated factorisation solves a random system to its precision
    (relative error below sqrt(n) eps cond(A), against LAPACK's FP64 solve),
    ragged last panel included."""
    rng = np.random.default_rng(3)
    n = 2 * S.PANEL + 29
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    B = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
    x = np.linalg.solve(A, B)
    y = S.BlockedLU(A, mode).solve(B.astype(np.complex64))
    err = np.linalg.norm(y - x) / np.linalg.norm(x)
    kappa = np.linalg.cond(A)
    assert err < np.sqrt(n) * eps * kappa
    if mode == "tf32":
        assert err > 2.0 ** -24 * kappa      # TF32 operands really were rounded


def _solve(problem, contour, m0, X0, norms, mode, sweeps):
    r, _, _ = S.run(problem, contour, m0, X0, mode, sweeps, 1e-10, 30, norms)
    return r


def test_low_precision_node_solves_reach_fp64_accuracy():
    """The n = 256 QEP and its stored circle (16 eigenvalues inside): FP32 and
    TF32 node solves, without refinement, converge like FP64."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "contours.json")))
    g = g["qep_plain_n256"]
    problem = config1_qep(256, 0)
    contour = {"center": complex(*g["center"]), "ra": g["ra"], "rb": g["rb"], "nc": g["nc"],
               "rule": g["rule"]}
    m0 = g["m0"]
    X0 = start_block(problem["n"], m0, 0)
    norms = O.term_norms(problem)
    ref = _solve(problem, contour, m0, X0, norms, "fp64", 0)
    assert ref["converged"] and ref["inside"].sum() == g["count"]
    lam_ref = ref["lam"][ref["inside"]]
    for mode, sweeps in (("fp32", 0), ("tf32", 0), ("tf32", 1)):
        r = _solve(problem, contour, m0, X0, norms, mode, sweeps)
        assert r["converged"], (mode, sweeps)
        assert r["iters"] <= ref["iters"] + 1, (mode, sweeps, r["iters"], ref["iters"])
        lam = r["lam"][r["inside"]]
        assert len(lam) == len(lam_ref)
        err = max(np.min(np.abs(lam_ref - l)) / abs(l) for l in lam)
        assert err < 1e-12, (mode, sweeps, err)


def test_planted_non_residual_filter_stalls_at_solve_precision(monkeypatch):
    """Planted mistake: Step 4 written as T(z_j)^{-1}(T(z_j) X - T(X, Lambda)),
    equal to X - T(z_j)^{-1} T(X, Lambda) in exact arithmetic, hands the
    solve a right-hand side that does not vanish; with TF32 node solves the
    iteration then stalls far above the tolerance."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "contours.json")))
    g = g["qep_plain_n256"]
    problem = config1_qep(256, 0)
    contour = {"center": complex(*g["center"]), "ra": g["ra"], "rb": g["rb"], "nc": g["nc"],
               "rule": g["rule"]}
    z, _ = O.quadrature(contour["center"], contour["ra"], contour["rb"], contour["nc"], "gl")

    def planted(lus, zz, omega, X, lam, R):
        Q = np.zeros_like(X)
        for solve, zj, wj in zip(lus, zz, omega):
            Q += solve(O.assemble(problem, zj) @ X - R) * (wj / (zj - lam))[None, :]
        return Q

    monkeypatch.setattr(O, "filter_update", planted)
    X0 = start_block(problem["n"], g["m0"], 0)
    r = _solve(problem, contour, g["m0"], X0, O.term_norms(problem), "tf32", 0)
    assert not r["converged"]
    assert min(r["history"][1:]) > 1e-8


def test_found_counts_reference_pairs_per_iteration():
    """The study's per-iteration count: a reference eigenvalue is found when a
    Ritz value with relres <= tol lies within tol (relative) of it."""
    ref = np.array([1.0 + 1.0j, 2.0 + 0.0j])
    trace = [(np.array([1.0 + 1.0j, 2.0 + 1e-6j]), np.array([1e-12, 1e-12])),   # 2+1e-6i too far
             (np.array([1.0 + 1.0j, 2.0 + 0.0j]), np.array([1e-9, 1e-12])),     # 1+1i residual too big
             (np.array([1.0 + 1.0j, 2.0 + 0.0j]), np.array([1e-12, 1e-12]))]
    assert S.found(trace, ref) == [1, 1, 2]
    assert S.found([(np.array([]), np.array([]))], ref) == [0]
