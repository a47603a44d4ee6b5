"""Parity of the CUDA library (through its C ABI) with the FP64 oracle."""
import json
import os

import numpy as np
import pytest

import oracle as O
from tests.closed_forms import (inside_mask, match_sets, load_table1, second_companion_eigs,
                                problem_mats, family_eigs)
from workloads import (mass_spring, config1_qep, random_pep, start_block, linear_problem,
                       closed_form_family)

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def lib():
    import paper_1801_09794_gb300 as P
    P.load_library()
    return P


def _contour_for(p, count, target=0.0):
    lam = second_companion_eigs(problem_mats(p))
    lam = lam[np.isfinite(lam)]
    c = lam[np.argmin(np.abs(lam - target))]
    d = np.sort(np.abs(lam - c))
    r = 0.5 * (d[count - 1] + d[count])
    return c, r, lam


def _relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ------------------------------------------------------------------ quadrature
@pytest.mark.parametrize("rule,nc", [("gl", 16), ("trapezoid", 12), ("gl_halves", 8), ("gl", 1)])
def test_nodes_match_oracle(lib, rule, nc):
    p = random_pep(40, 2, seed=1)
    s = lib.FeastNL(p, "fp64")
    s.set_contour(0.1 + 0.2j, 0.7, 0.4, nc, rule)
    z, w = s.get_nodes()
    zo, wo = O.quadrature(0.1 + 0.2j, 0.7, 0.4, nc, rule)
    assert np.max(np.abs(z - zo)) < 1e-14 and np.max(np.abs(w - wo)) < 1e-14
    s.close()


# ------------------------------------------------------------------ node LU + solve
@pytest.mark.parametrize("prec,n", [("fp64", 150), ("fp32", 150), ("fp64", 33), ("fp32", 200),
                                    ("fp64", 1), ("fp32", 65), ("fp32", 1), ("fp32", 700),
                                    # odd orders: one ragged panel, a ragged pair, and
                                    # a first panel taller than one CTA's 1024 rows
                                    ("fp32", 3), ("fp32", 17), ("fp64", 127), ("fp32", 127),
                                    ("fp32", 1027)])
def test_node_solve_matches_oracle(lib, prec, n):
    p = random_pep(n, 2, seed=3)
    c, ra = 0.05 + 0.1j, 0.6
    s = lib.FeastNL(p, prec)
    s.set_contour(c, ra, ra, 6, "gl")
    z, _ = O.quadrature(c, ra, ra, 6, "gl")
    rng = np.random.default_rng(7)
    nrhs = 96 if n >= 500 else 5        # 96: several row tiles and two column tiles
    R = rng.standard_normal((n, nrhs)) + 1j * rng.standard_normal((n, nrhs))
    for j in range(6):
        T = O.assemble(p, z[j])
        ref = np.linalg.solve(T, R)
        got = s.node_solve(j, R)
        kappa = np.linalg.cond(T)
        tol = (1e-14 if prec == "fp64" else 1e-6) * max(kappa, 10.0) * max(1.0, np.sqrt(n) / 4)
        assert _relerr(got, ref) < tol, (j, _relerr(got, ref), kappa)
    s.close()


@pytest.mark.parametrize("n", [1500, 4096])
def test_panel_cluster_factors_bit_identical(lib, n, monkeypatch):
    """A complex64 panel spread over a cluster of CTAs (several shapes) gives
    the same factors, bit for bit, as the panel on one CTA: the node solves
    through them agree exactly."""
    p = random_pep(n, 2, seed=11)
    rng = np.random.default_rng(5)
    R = rng.standard_normal((n, 24)) + 1j * rng.standard_normal((n, 24))
    out = {}
    for rpc in ("0", "512", "1024", "300"):
        monkeypatch.setenv("FEAST_NL_PANEL_ROWS_PER_CTA", rpc)
        s = lib.FeastNL(p, "fp32")
        s.set_contour(0.05 + 0.1j, 0.6, 0.6, 4, "gl")
        out[rpc] = [s.node_solve(j, R) for j in range(4)]
        s.close()
    for rpc in ("512", "1024", "300"):
        for j in range(4):
            assert np.array_equal(out[rpc][j], out["0"][j]), (rpc, j)


# ------------------------------------------------------------------ Step 4 and Step 1 pieces
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_i8"])
def test_filter_apply_matches_oracle(lib, prec):
    n, m = 170, 9
    p = random_pep(n, 2, seed=5)
    c, ra, rb = -0.1 + 0.05j, 0.5, 0.3
    s = lib.FeastNL(p, prec)
    s.set_contour(c, ra, rb, 8, "gl")
    z, w = O.quadrature(c, ra, rb, 8, "gl")
    lus = O.factor_nodes(p, z)
    rng = np.random.default_rng(11)
    X = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    X /= np.linalg.norm(X, axis=0)
    lam = c + 0.4 * (rng.standard_normal(m) + 1j * rng.standard_normal(m))
    R = O.block_residual(p, X, lam)
    ref = O.filter_update(lus, z, w, X, lam, R)
    got = s.filter_apply(X, lam)
    kappa = max(np.linalg.cond(O.assemble(p, zj)) for zj in z)
    tol = 1e-12 * kappa if prec == "fp64" else 2e-6 * kappa    # FP32 node solves otherwise
    assert _relerr(got, ref) < tol
    s.close()


@pytest.mark.parametrize("prec,n,m", [("fp64", 190, 12), ("fp32_i8", 190, 12),
                                      ("fp32_i8", 300, 40), ("fp32_i8", 1, 1)])
def test_project_matches_oracle(lib, prec, n, m):
    p = random_pep(n, 3, seed=8)
    s = lib.FeastNL(p, prec)
    Q = O.orthonormalize(start_block(n, m, 3))
    got = s.project(Q, 3)
    ref = O.projected_coefficients(p, Q)
    for gp, rp in zip(got, ref):
        assert _relerr(gp, rp) < 1e-13
    s.close()


@pytest.mark.parametrize("prec", ["fp32_i8", "fp32"])
def test_project_with_diagonal_terms(lib, prec):
    """Dense coefficients that are diagonal (a non-identity mass matrix) take
    the diagonal-scaling path for A_t Q in the digit-split precision; the
    projections and a whole solve still match the oracle."""
    n, m = 300, 24
    rng = np.random.default_rng(21)
    p = random_pep(n, 2, seed=9)
    p["terms"][2]["A"] = np.diag(1.0 + 0.1 * rng.uniform(size=n)).astype(np.complex128)
    p["terms"][0]["A"] = np.diag(rng.standard_normal(n) + 1j * rng.standard_normal(n))
    s = lib.FeastNL(p, prec)
    Q = O.orthonormalize(start_block(n, m, 3))
    got = s.project(Q, 2)
    ref = O.projected_coefficients(p, Q)
    for gp, rp in zip(got, ref):
        assert _relerr(gp, rp) < 1e-13
    lam_all = O.brute_force_eigs(p)
    lam_all = lam_all[np.isfinite(lam_all)]
    c = lam_all[np.argmin(np.abs(lam_all - 0.3j))]
    d = np.sort(np.abs(lam_all - c))
    r = 0.5 * (d[5] + d[6])
    s.set_contour(c, r, r, 16, "gl")
    s.solve(32, tol=1e-12, maxit=60, X0=start_block(n, 32, 4), allow=(lib.FEAST_NL_ENOT_CONVERGED,))
    lam, _, rr = s.get_eigpairs(inside_only=True)
    want = lam_all[np.abs(lam_all - c) < r]
    assert len(lam) == len(want) == 6
    assert match_sets(lam, want) < 1e-10 and np.all(rr <= 1e-10)
    s.close()


def test_project_matches_oracle_n4096(lib):
    """Projections at the largest K of the digit-split products (n = 4096,
    K = 2n = 8192 in the real embedding) on the n = 4096 QEP with m0 = 96,
    against FP64.  Seven 7-bit digit slices keep 49 bits of each entry relative
    to its row's largest entry; the stiffness matrix K has diagonal entries
    near 50 and off-diagonal entries near 1, so its off-diagonal entries keep
    ~43 bits in W = K Q: 2^-43 = 1.1e-13 relative, the level measured here.
    Tolerance 1e-12 (the worst-case FP32 accumulation bound of the low levels
    would allow 6e-11)."""
    from workloads import config2_qep
    p = config2_qep(4096, 0)
    s = lib.FeastNL(p, "fp32_i8")
    Q = O.orthonormalize(start_block(4096, 96, 5))
    got = s.project(Q, 2)
    ref = O.projected_coefficients(p, Q)
    errs = [_relerr(gp, rp) for gp, rp in zip(got, ref)]
    print("projection errors at n = 4096, m0 = 96:", ", ".join("%.2e" % e for e in errs))
    assert max(errs) < 1e-12, errs
    s.close()


# ------------------------------------------------------------------ whole solve
def test_qep_mixed_n4096_matches_stored_reference(lib):
    """The n = 4096 QEP with 16 nodes and m0 = 96 in the default mixed precision,
    through the C ABI as a user calls it: every one of the 64 eigenvalues the
    oracle's shift-invert Arnoldi found inside the circle (stored), to 1e-10
    relative, and every residual <= 1e-10 (Algorithm 1, Step 3)."""
    from workloads import config2_qep
    with open(os.path.join(GOLD, "contours.json")) as f:
        w = json.load(f)["qep_mixed_n4096"]
    gold = np.array([complex(*x) for x in w["eigs_inside"]])
    p = config2_qep(4096, 0)
    s = lib.FeastNL(p, "fp32_i8")
    s.set_contour(complex(*w["center"]), w["ra"], w["rb"], w["nc"], w["rule"])
    st, info = s.solve(w["m0"], tol=1e-10, maxit=40, seed=0)
    lam, X, rr = s.get_eigpairs(inside_only=True, vectors=False)
    assert info.n_inside == len(lam) == len(gold) == w["count"] == 64
    err = match_sets(lam, gold)
    print(f"n = 4096 QEP: {info.iters} iterations, max rel eigenvalue error {err:.2e}, "
          f"max relres {np.max(rr):.2e}")
    assert err < 1e-10
    assert np.all(rr <= 1e-10)
    s.close()
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_i8"])
def test_solve_example1_table1(lib, prec):
    rows = load_table1(os.path.join(GOLD, "e1_table1.txt"))
    p = mass_spring(1000, 0.6202, 0.4807)
    s = lib.FeastNL(p, prec)
    s.set_contour(-1.55, 0.05, 0.0035, 16, "gl")
    st, info = s.solve(22, tol=1e-10, maxit=20, X0=start_block(1000, 22, 0))
    lam, X, rr = s.get_eigpairs(inside_only=True)
    assert info.n_inside == 20 and len(lam) == 20
    assert np.max(np.abs(np.sort(lam.real) - np.sort([r[1] for r in rows]))) < 6e-11
    assert np.max(np.abs(lam.imag)) < 1e-11
    assert np.all(rr <= 1e-10)
    if prec == "fp64":
        assert info.iters == 3          # the paper's "three FEAST iterations"
    # the returned pairs meet Step 3's stopping test when it is re-evaluated on
    # the host (FP64, power-iteration norms), up to the host's own rounding
    R = O.block_residual(p, X, lam)
    rr_host = O.relative_residuals(p, R, lam, O.term_norms(p))
    assert np.all(rr_host <= 1.01e-10), rr_host.max()
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_i8"])
def test_solve_plain_qep_matches_oracle(lib, prec):
    with open(os.path.join(GOLD, "contours.json")) as f:
        w = json.load(f)["qep_plain_n256"]
    p = config1_qep(256, 0)
    c = complex(*w["center"])
    X0 = start_block(256, 24, 0)
    ref = O.nlfeast(p, {"center": c, "ra": w["ra"], "rb": w["rb"], "nc": 8, "rule": "gl"}, 24, X0,
                    tol=1e-12, maxit=60)
    assert ref["converged"]
    s = lib.FeastNL(p, prec)
    s.set_contour(c, w["ra"], w["rb"], 8, "gl")
    st, info = s.solve(24, tol=1e-10, maxit=60, X0=X0)
    lam, X, rr = s.get_eigpairs(inside_only=True)
    gold = np.array([complex(*x) for x in w["eigs_inside"]])
    assert len(lam) == 16 and info.n_converged == 16
    assert match_sets(lam, ref["lam"][ref["inside"]]) < 1e-10
    assert match_sets(lam, gold) < 1e-10
    assert np.all(rr <= 1e-10)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_i8"])
def test_iteration_graph_equals_eager(lib, prec):
    # the captured iteration replays exactly the launches of the eager loop
    with open(os.path.join(GOLD, "contours.json")) as f:
        w = json.load(f)["qep_plain_n256"]
    p = config1_qep(256, 0)
    c = complex(*w["center"])
    X0 = start_block(256, 24, 0)
    out = []
    for graph in (False, True, False):        # the first run fills the solve autotuner's cache
        s = lib.FeastNL(p, prec)
        s.set_iteration_graph(graph)
        s.set_contour(c, w["ra"], w["rb"], 8, "gl")
        l0 = lib.launch_count()
        st, info = s.solve(24, tol=1e-10, maxit=60, X0=X0)
        launches = lib.launch_count() - l0
        lam, X, rr = s.get_eigpairs(inside_only=True)
        out.append((info.iters, launches, lam, X, rr))
        s.close()
    (i1, n1, l1, x1, r1), (i2, n2, l2, x2, r2) = out[1:]
    assert i1 == i2 and i1 > 2 and n1 == n2
    assert np.array_equal(l1, l2) and np.array_equal(x1, x2) and np.array_equal(r1, r2)


@pytest.mark.parametrize("k,prec", [(3, "fp64"), (3, "fp32"), (1, "fp32"), (3, "fp32_i8")])
def test_solve_random_pep_matches_bruteforce(lib, k, prec):
    n = 130 if k > 1 else 150
    p = random_pep(n, k, seed=20 + k) if k > 1 else linear_problem(n, seed=4)
    c, r, lam_all = _contour_for(p, 7, target=0.3 + 0.2j)
    # m0 = 14 makes the oracle itself oscillate on the cubic case; 20 converges
    m0 = 20 if k == 3 else 14
    X0 = start_block(n, m0, 9)
    orc = O.nlfeast(p, {"center": c, "ra": r, "rb": r, "nc": 16, "rule": "gl"}, m0, X0,
                    tol=1e-12, maxit=80)
    assert orc["converged"]
    s = lib.FeastNL(p, prec)
    s.set_contour(c, r, r, 16, "gl")
    st, info = s.solve(m0, tol=1e-12, maxit=80, X0=X0)
    lam, X, rr = s.get_eigpairs(inside_only=True)
    ref = lam_all[inside_mask(lam_all, c, r, r)]
    assert match_sets(lam, orc["lam"][orc["inside"]]) < 1e-10
    assert len(lam) == len(ref) == 7
    assert match_sets(lam, ref) < 1e-10
    assert np.all(rr <= 1e-10)
    s.close()


def test_solve_max_m0_closed_form(lib):
    """m0 at its maximum (112) on a quadratic with closed-form eigenvalues
    (A2 = I, A1 = 0.1 I, A0 = tridiag(-1, 3, -1): lambda = -0.05 +- i sqrt(s - 0.0025)
    for the tridiagonal's eigenvalues s).  The reduced companion matrix (224 x 224)
    no longer fits in shared memory: the QR chase runs on the global copy and the
    Hessenberg reduction keeps only its trailing columns on chip."""
    n, m0, cnt = 200, 112, 56
    c, d, a = [0.0, 0.1, 1.0], [1.0, 0.0, 0.0], 3.0
    p = closed_form_family(n, c, d, a)
    lam_all = family_eigs(n, c, d, a)
    cen = -0.05 + 1.6j
    dist = np.sort(np.abs(lam_all - cen))
    r = 0.5 * (dist[cnt - 1] + dist[cnt])       # boundary midway between two eigenvalues
    s = lib.FeastNL(p, "fp32_i8")
    s.set_contour(cen, r, r, 16, "gl")
    st, info = s.solve(m0, tol=1e-11, maxit=60, X0=start_block(n, m0, 3))
    lam, X, rr = s.get_eigpairs(inside_only=True)
    ref = lam_all[inside_mask(lam_all, cen, r, r)]
    assert len(lam) == len(ref) == cnt
    assert match_sets(lam, ref) < 1e-10
    assert np.all(rr <= 1e-11)
    s.close()


def test_device_random_start_converges(lib):
    p = random_pep(120, 2, seed=31)
    c, r, lam_all = _contour_for(p, 5, target=-0.2)
    s = lib.FeastNL(p, "fp32")
    s.set_contour(c, r, r, 16, "trapezoid")
    st, info = s.solve(10, tol=1e-12, maxit=80, seed=123)      # X0 drawn on the device
    lam, X, rr = s.get_eigpairs(inside_only=True)
    assert match_sets(lam, lam_all[inside_mask(lam_all, c, r, r)]) < 1e-10
    s.close()


# ------------------------------------------------------------------ edge cases
def test_singular_node_reported(lib):
    n = 20
    probe = lib.FeastNL(linear_problem(n, seed=1), "fp64")
    probe.set_contour(0.0, 1.0, 1.0, 4, "trapezoid")
    z, _ = probe.get_nodes()
    probe.close()
    d = np.linspace(-3, 3, n).astype(np.complex128)
    d[5] = z[2]                          # T(z_2) = diag(d) - z_2 I has an exact zero
    p = {"n": n, "terms": [{"kind": "pow", "p": 0, "scale": 1.0, "A": np.diag(d)},
                           {"kind": "pow", "p": 1, "scale": -1.0, "A": None}]}
    s = lib.FeastNL(p, "fp64")
    with pytest.raises(lib.FeastError) as ei:
        s.set_contour(0.0, 1.0, 1.0, 4, "trapezoid")
    assert ei.value.status == lib.FEAST_NL_ESINGULAR_NODE
    s.close()


def test_too_small_subspace_reported(lib):
    p = random_pep(100, 2, seed=2)
    c, r, _ = _contour_for(p, 12)
    s = lib.FeastNL(p, "fp32")
    s.set_contour(c, r, r, 8, "gl")
    st, info = s.solve(6, tol=1e-10, maxit=6, X0=start_block(100, 6, 1),
                       allow=(lib.FEAST_NL_ETOO_MANY, lib.FEAST_NL_ENOT_CONVERGED))
    assert st in (lib.FEAST_NL_ETOO_MANY, lib.FEAST_NL_ENOT_CONVERGED)
    lam, X, rr = s.get_eigpairs()
    assert len(lam) == 6 and np.all(np.isfinite(lam))
    s.close()


def test_invalid_arguments_rejected(lib):
    p = random_pep(30, 2, seed=2)
    s = lib.FeastNL(p, "fp64")
    for args in [(0.0, -1.0, 1.0, 8, "gl"), (0.0, 1.0, 1.0, 0, "gl"), (0.0, 1.0, 1.0, 7, "gl_halves")]:
        with pytest.raises(lib.FeastError) as ei:
            s.set_contour(*args)
        assert ei.value.status == lib.FEAST_NL_EINVAL
    with pytest.raises(lib.FeastError) as ei:
        s.solve(8)                               # no contour yet
    assert ei.value.status == lib.FEAST_NL_EINVAL
    s.set_contour(0.0, 0.5, 0.5, 8, "gl")
    for m0 in (0, 31, 113):
        with pytest.raises(lib.FeastError) as ei:
            s.solve(m0)
        assert ei.value.status == lib.FEAST_NL_EINVAL
    s.close()


def test_device_pointers_roundtrip(lib):
    torch = pytest.importorskip("torch")
    n = 90
    p = random_pep(n, 2, seed=12)
    pd = {"n": n, "terms": [dict(t, A=torch.from_numpy(t["A"]).cuda()) for t in p["terms"]]}
    c, r, lam_all = _contour_for(p, 4, target=0.1)
    s = lib.FeastNL(pd, "fp64")
    s.set_contour(c, r, r, 16, "gl")
    X0 = torch.from_numpy(start_block(n, 8, 2)).cuda()
    s.solve(8, tol=1e-12, maxit=60, X0=X0)
    lam, X, rr = s.get_eigpairs(inside_only=True)
    assert match_sets(lam, lam_all[inside_mask(lam_all, c, r, r)]) < 1e-10
    s.close()
