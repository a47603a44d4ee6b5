"""Spectrum slicing through the C ABI (Sec. 1 and Sec. 3: disjoint regions of the
plane are solved independently): many contours of one problem, their node
matrices factored in one batch and their iterations run together, against QZ,
against one-contour solves, with and without the iteration graph, and at full
size (n = 2048 cubic, 64 discs) against the stored references."""
import json
import os

import numpy as np
import pytest

from tests.closed_forms import inside_mask, match_sets, problem_mats, second_companion_eigs
from workloads import cubic_pep, random_pep

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "contours.json")
TARGETS = [0.35 + 0.2j, -0.4 + 0.5j, 0.6 - 0.6j, -0.8 - 0.3j, 1.2 + 0.1j, 0.0 - 1.1j]


@pytest.fixture(scope="module")
def lib():
    import paper_1801_09794_gb300 as P
    P.load_library()
    return P


@pytest.fixture(scope="module")
def small():
    """Random cubic n = 120 and six discs around eigenvalues near TARGETS, each
    with its radius in the middle of the gap after the 5th nearest eigenvalue."""
    p = random_pep(120, 3, seed=31)
    lam = second_companion_eigs(problem_mats(p))
    lam = lam[np.isfinite(lam)]
    centers, radii = [], []
    for t in TARGETS:
        c = lam[np.argmin(np.abs(lam - t))]
        d = np.sort(np.abs(lam - c))
        centers.append(c)
        radii.append(0.5 * (d[4] + d[5]))
    return p, lam, np.array(centers), np.array(radii)


# Subspace per disc: 24 for 5 eigenvalues inside.  Rayleigh-Ritz on the cubic
# now and then keeps a spurious Ritz value inside a disc for many iterations;
# the FP64 oracle takes 5 to 18 iterations over these discs and three starts
# with 16 columns, 4 to 9 with 24, so 24 keeps every solve far below maxit.
M0 = 24


def _solve(lib, p, centers, radii, prec, graph=True, m0=M0, nc=16, tol=1e-12, maxit=80, seed=5):
    s = lib.FeastNL(p, prec)
    sl = lib.Slices(s, centers, radii, radii, nc, "gl")
    st, infos = sl.solve(m0, tol=tol, maxit=maxit, seed=seed, graph=graph)
    out = [sl.get_eigpairs(d, inside_only=True) for d in range(len(centers))]
    iters = [i.iters for i in infos]
    sl.close()
    s.close()
    return st, iters, out


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_i8"])
def test_slices_match_qz(lib, small, prec):
    p, lam_all, centers, radii = small
    st, iters, out = _solve(lib, p, centers, radii, prec)
    assert st == lib.FEAST_NL_OK
    for c, r, (lam, X, rr) in zip(centers, radii, out):
        ref = lam_all[inside_mask(lam_all, c, r, r)]
        assert len(lam) == len(ref) == 5
        assert match_sets(lam, ref) < 1e-10
        assert np.all(rr <= 1e-12)
        # unit Ritz vectors
        assert np.allclose(np.linalg.norm(X, axis=0), 1.0, atol=1e-12)


@pytest.mark.parametrize("prec", ["fp32", "fp32_i8"])
def test_slices_graph_equals_eager(lib, small, prec):
    # the captured graph replays exactly the launches of the eager iteration
    p, _, centers, radii = small
    st1, it1, g = _solve(lib, p, centers, radii, prec, graph=True)
    st2, it2, e = _solve(lib, p, centers, radii, prec, graph=False)
    assert st1 == st2 == lib.FEAST_NL_OK and it1 == it2
    for (l1, x1, r1), (l2, x2, r2) in zip(g, e):
        assert np.array_equal(l1, l2) and np.array_equal(x1, x2) and np.array_equal(r1, r2)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_i8"])
def test_first_slice_equals_single_contour_solve(lib, small, prec):
    # contour 0 of a set starts from the same device-drawn block as a one-contour
    # solve with the same seed; every per-contour product is the same arithmetic
    p, _, centers, radii = small
    st, iters, out = _solve(lib, p, centers, radii, prec, seed=8)
    s = lib.FeastNL(p, prec)
    s.set_contour(centers[0], radii[0], radii[0], 16, "gl")
    st1, info = s.solve(M0, tol=1e-12, maxit=80, seed=8)
    lam1, X1, rr1 = s.get_eigpairs(inside_only=True)
    s.close()
    assert info.iters == iters[0]
    lam0, X0, rr0 = out[0]
    if prec == "fp32_i8":
        # the digit-split product tiles the columns of all contours together
        assert match_sets(lam0, lam1) < 1e-12
    else:
        assert np.array_equal(lam0, lam1) and np.array_equal(rr0, rr1)


def test_slices_invalid_arguments(lib, small):
    p, _, centers, radii = small
    s = lib.FeastNL(p, "fp32")
    with pytest.raises(lib.FeastError):
        lib.Slices(s, centers, -radii, radii, 8)
    with pytest.raises(lib.FeastError):
        lib.Slices(s, centers, radii, radii, 0)
    sl = lib.Slices(s, centers[:2], radii[:2], radii[:2], 8)
    with pytest.raises(lib.FeastError):
        sl.get_eigpairs(0)                     # nothing solved yet
    with pytest.raises(lib.FeastError):
        sl.solve(200)                          # m0 above the reduced solver's limit
    sl.solve(16, tol=1e-10, maxit=40, allow=(lib.FEAST_NL_ENOT_CONVERGED,))
    with pytest.raises(lib.FeastError):
        sl.get_eigpairs(2)                     # no such contour
    sl.close()
    s.close()


def test_slices_full_size_match_stored_eigenvalues(lib):
    """The benchmark workload: cubic n = 2048, 64 discs, 8 nodes each (512
    node LUs in one batch), m0 = 16."""
    g = json.load(open(GOLDEN))["slices_n2048"]
    p = cubic_pep(2048, 0)
    centers = np.array([complex(*c) for c in g["centers"]])
    s = lib.FeastNL(p, "fp32_i8")
    sl = lib.Slices(s, centers, g["r"], g["r"], g["nc"], g["rule"])
    # stopping at relres 1e-12: these non-normal eigenvalues (condition ~5) need it
    # for 1e-10 eigenvalue accuracy, as the oracle itself does
    st, infos = sl.solve(g["m0"], tol=1e-12, maxit=60, seed=0)
    assert st == lib.FEAST_NL_OK, [i.status for i in infos]
    found = 0
    for d, c in enumerate(centers):
        lam, X, rr = sl.get_eigpairs(d, inside_only=True, vectors=False)
        ref = np.array([complex(*e) for e in g["eigs_inside"][d]])
        assert len(lam) == len(ref), (d, len(lam), len(ref))
        if len(ref):
            assert match_sets(lam, ref) < 1e-10
        assert np.all(rr <= 1e-10)
        found += len(lam)
    assert found == g["count"]
    sl.close()
    s.close()
