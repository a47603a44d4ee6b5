"""Non-polynomial T (the delay problem) through the C ABI: the closed-form
Lambert-W spectrum of a structured family and parity with the FP64 oracle on
a random delay problem."""
import numpy as np
import pytest

import oracle as O
from tests.closed_forms import delay_family_eigs, inside_mask, match_sets
from workloads import delay_family, delay_problem, start_block

pytestmark = pytest.mark.gpu

FAM = dict(n=30, c=[-1.0, 0.3], d=[0.5, 0.1], a=2.0, tau=1.0)


@pytest.fixture(scope="module")
def lib():
    import paper_1801_09794_gb300 as P
    P.load_library()
    return P


def _host_relres(p, lam, X):
    R = O.block_residual(p, X, lam)
    return O.relative_residuals(p, R, lam, O.term_norms(p))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_i8"])
def test_delay_family_matches_lambert_w(lib, prec):
    lam_all = delay_family_eigs(FAM["n"], FAM["c"], FAM["d"], FAM["a"], FAM["tau"])
    real0 = np.sort(lam_all[np.abs(lam_all.imag) < 1e-12].real)
    c = complex(0.5 * (real0[10] + real0[3]))
    r = float(0.5 * (real0[10] - real0[3]) + 1e-3)
    ref = lam_all[inside_mask(lam_all, c, r, r)]
    p = delay_family(**FAM)
    s = lib.FeastNL(p, prec)
    s.set_contour(c, r, r, 16, "gl")
    st, info = s.solve(12, tol=1e-11, maxit=30, X0=start_block(FAM["n"], 12, 3))
    lam, X, rr = s.get_eigpairs(inside_only=True)
    assert len(lam) == len(ref) == 8
    assert match_sets(lam, ref) < 1e-10
    assert np.all(rr <= 1e-11)
    assert np.all(_host_relres(p, lam, X) <= 1.01e-11)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_random_delay_matches_oracle(lib, prec):
    n, m0 = 120, 24
    p = delay_problem(n, 0)
    contour = {"center": -0.99 + 0j, "ra": 0.5, "rb": 0.25, "nc": 24, "rule": "gl"}
    X0 = start_block(n, m0, 1)
    ref = O.nlfeast(p, contour, m0, X0, tol=1e-10, maxit=40)
    assert ref["converged"]
    lam_ref = ref["lam"][ref["inside"]]
    assert len(lam_ref) == O.winding_count(p, contour["center"], 0.5, 0.25, 512) == 16
    s = lib.FeastNL(p, prec)
    s.set_contour(contour["center"], 0.5, 0.25, 24, "gl")
    st, info = s.solve(m0, tol=1e-10, maxit=40, X0=X0)
    lam, X, rr = s.get_eigpairs(inside_only=True)
    assert len(lam) == len(lam_ref)
    assert match_sets(lam, lam_ref) < 1e-10
    assert np.all(_host_relres(p, lam, X) <= 1.01e-10)
    s.close()


def test_delay_m0_limit(lib):
    p = delay_problem(80, 1)
    s = lib.FeastNL(p, "fp32")
    s.set_contour(-1.0 + 0j, 0.5, 0.25, 8, "gl")
    with pytest.raises(lib.FeastError) as e:
        s.solve(65, tol=1e-10, maxit=2)
    assert e.value.status == lib.FEAST_NL_EINVAL
    s.close()


def test_delay_n2048_matches_stored_reference(lib):
    """The full-size delay workload: every eigenvalue the stored oracle solve found
    inside the ellipse (29, argument-principle count 29), to 1e-10."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "contours.json")) as f:
        w = json.load(f)["delay_n2048"]
    gold = np.array([complex(*x) for x in w["eigs_inside"]])
    p = delay_problem(2048, 0)
    s = lib.FeastNL(p, "fp32_i8")
    s.set_contour(complex(*w["center"]), w["ra"], w["rb"], w["nc"], w["rule"])
    st, info = s.solve(w["m0"], tol=1e-10, maxit=40, seed=0)
    lam, X, rr = s.get_eigpairs(inside_only=True, vectors=False)
    assert len(lam) == len(gold) == w["winding_count"]
    assert match_sets(lam, gold) < 1e-10
    assert np.all(rr <= 1e-10)
    # The iteration count of this workload is set by spurious Ritz values of the
    # projected problem: the 29 eigenvalues converge within ~5 iterations, but
    # a Ritz value of Q^H T Q that matches no eigenvalue of T can sit inside C
    # with a residual near 1e-3 for several iterations, and the test passes
    # once it leaves (the largest residual then drops from ~1e-3 to ~1e-16 in
    # one step).  The FP64 oracle takes 6, 6, 17 and 6 iterations from four
    # start blocks (9 on the GPU host's Arm cores from the bench's start); the
    # GPU path takes 7 (it has taken 10 and 14 with earlier rounding).  The
    # bound is the oracle's 9 plus two: a mixed-precision path that converges
    # more slowly than the FP64 algorithm fails here.
    assert info.iters <= 11, info.iters
    s.close()
