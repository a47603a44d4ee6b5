"""Grouped factorisation through the C ABI: the node matrices of several
problems of different orders (one contour each) factored in one launch
sequence per panel, then each problem solved on its own handle; results
against QZ and against the same problems factored one by one."""
import numpy as np
import pytest

from tests.closed_forms import inside_mask, match_sets, problem_mats, second_companion_eigs
from workloads import random_pep, start_block

pytestmark = pytest.mark.gpu

# (n, degree, seed): orders that are and are not multiples of the 64-column panel
CASES = [(130, 3, 21), (256, 2, 5), (200, 3, 8)]
# Subspace size: 32 for 7 eigenvalues inside.  With 20, Rayleigh-Ritz on the
# cubic (60 Ritz values for 20 columns) now and then puts a spurious Ritz value
# inside the contour whose residual never falls, and the iteration count
# becomes erratic: the FP64 oracle itself takes 79 iterations on the n = 130
# problem from this start (6 to over 80 over m0 = 16 .. 28 and three starts),
# against 4 to 15 with m0 = 32 over six starts for all three problems.
M0 = 32


@pytest.fixture(scope="module")
def lib():
    import paper_1801_09794_gb300 as P
    P.load_library()
    return P


@pytest.fixture(scope="module")
def problems():
    out = []
    for n, k, seed in CASES:
        p = random_pep(n, k, seed)
        lam = second_companion_eigs(problem_mats(p))
        lam = lam[np.isfinite(lam)]
        c = lam[np.argmin(np.abs(lam - (0.3 + 0.2j)))]
        d = np.sort(np.abs(lam - c))
        r = 0.5 * (d[6] + d[7])                  # 7 inside
        out.append((p, lam, c, r))
    return out


@pytest.mark.parametrize("prec", ["fp32", "fp32_i8"])
def test_group_solves_match_qz(lib, problems, prec):
    hs = [lib.FeastNL(p, prec) for p, _, _, _ in problems]
    lib.set_contour_group(hs, [c for _, _, c, _ in problems], [r for _, _, _, r in problems],
                          [r for _, _, _, r in problems], 16)
    for h, (p, lam_all, c, r) in zip(hs, problems):
        st, info = h.solve(M0, tol=1e-12, maxit=80, X0=start_block(p["n"], M0, 9))
        lam, X, rr = h.get_eigpairs(inside_only=True)
        ref = lam_all[inside_mask(lam_all, c, r, r)]
        assert len(lam) == len(ref) == 7
        assert match_sets(lam, ref) < 1e-10
        assert np.all(rr <= 1e-10)
        h.close()


def test_group_factors_match_one_by_one(lib, problems):
    # same node matrices and the same per-node kernel variants: the factors,
    # hence node solves and whole solves, are bit for bit those of a
    # factorisation of each problem on its own
    grouped = [lib.FeastNL(p, "fp32") for p, _, _, _ in problems]
    lib.set_contour_group(grouped, [c for _, _, c, _ in problems], [r for _, _, _, r in problems],
                          [r for _, _, _, r in problems], 16)
    rng = np.random.default_rng(3)
    for g, (p, _, c, r) in zip(grouped, problems):
        s = lib.FeastNL(p, "fp32")
        s.set_contour(c, r, r, 16)
        R = rng.standard_normal((p["n"], 4)) + 1j * rng.standard_normal((p["n"], 4))
        for j in (0, 7, 15):
            y1, y2 = g.node_solve(j, R), s.node_solve(j, R)
            assert np.array_equal(y1, y2)
        X0 = start_block(p["n"], M0, 4)
        g.solve(M0, tol=1e-12, maxit=80, X0=X0)
        s.solve(M0, tol=1e-12, maxit=80, X0=X0)
        l1, x1, r1 = g.get_eigpairs(inside_only=True)
        l2, x2, r2 = s.get_eigpairs(inside_only=True)
        assert np.array_equal(l1, l2) and np.array_equal(x1, x2) and np.array_equal(r1, r2)
        s.close()
        g.close()


@pytest.mark.parametrize("persistent", ["0", "1"])
def test_group_factors_match_one_by_one_either_path(lib, problems, persistent, monkeypatch):
    """The grouped factorisation by launches per panel step and by one
    persistent launch over all nodes (a device work queue) give the factors
    of the one-by-one factorisation (launches per step), bit for bit."""
    rng = np.random.default_rng(4)
    monkeypatch.setenv("FEAST_NL_LU_PERSISTENT", persistent)
    grouped = [lib.FeastNL(p, "fp32") for p, _, _, _ in problems]
    lib.set_contour_group(grouped, [c for _, _, c, _ in problems], [r for _, _, _, r in problems],
                          [r for _, _, _, r in problems], 16)
    monkeypatch.setenv("FEAST_NL_LU_PERSISTENT", "0")
    for g, (p, _, c, r) in zip(grouped, problems):
        s = lib.FeastNL(p, "fp32")
        s.set_contour(c, r, r, 16)
        R = rng.standard_normal((p["n"], 5)) + 1j * rng.standard_normal((p["n"], 5))
        for j in range(16):
            assert np.array_equal(g.node_solve(j, R), s.node_solve(j, R)), j
        s.close()
        g.close()


@pytest.mark.parametrize("n,nodes", [(700, 6), (1500, 4), (2048, 3)])
def test_persistent_factorisation_bit_identical(lib, n, nodes, monkeypatch):
    """One problem's node matrices factored by one persistent launch equal,
    bit for bit, those factored by launches per panel step with cluster
    panels and prioritised streams."""
    p = random_pep(n, 2, seed=17)
    rng = np.random.default_rng(8)
    R = rng.standard_normal((n, 12)) + 1j * rng.standard_normal((n, 12))
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("FEAST_NL_LU_PERSISTENT", mode)
        s = lib.FeastNL(p, "fp32")
        s.set_contour(0.05 + 0.1j, 0.6, 0.6, nodes, "gl")
        out[mode] = [s.node_solve(j, R) for j in range(nodes)]
        s.close()
    for j in range(nodes):
        assert np.array_equal(out["0"][j], out["1"][j]), j


def test_group_invalid_arguments(lib, problems):
    p = problems[0][0]
    a, b = lib.FeastNL(p, "fp32"), lib.FeastNL(p, "fp64")
    with pytest.raises(lib.FeastError):
        lib.set_contour_group([a, b], [0.1, 0.1], 0.2, 0.2, 8)        # complex128 factors
    with pytest.raises(lib.FeastError):
        lib.set_contour_group([a, a], [0.1, 0.1], 0.2, 0.2, 8)        # same handle twice
    with pytest.raises(lib.FeastError):
        lib.set_contour_group([a], [0.1], -0.2, 0.2, 8)               # bad radius
    a.close()
    b.close()
