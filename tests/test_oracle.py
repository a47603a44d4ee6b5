"""Pins of the FP64 oracle against values the paper prints, closed forms,
invariants and brute force (CPU only)."""
import os

import numpy as np
import pytest

import oracle.nlfeast_ref as O
from workloads import (mass_spring, closed_form_family, random_pep, linear_problem,
                       start_block, tridiag)
from tests.closed_forms import (family_eigs, second_companion_eigs, problem_mats,
                                inside_mask, match_sets, load_table1)

GOLD = os.path.join(os.path.dirname(__file__), "golden")
E1_CONTOUR = {"center": -1.55, "ra": 0.05, "rb": 0.0035, "nc": 16, "rule": "gl"}


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("rule", ["gl", "trapezoid", "gl_halves"])
def test_filter_is_one_at_circle_center(rule):
    c = 0.3 - 1.2j
    z, w = O.quadrature(c, 0.7, 0.7, 16, rule)
    assert abs(O.filter_function(c, z, w)[0] - 1.0) < 1e-14


def test_trapezoid_moments_vanish():
    c, r, nc = 1.0 + 2.0j, 0.5, 12
    z, w = O.quadrature(c, r, r, nc, "trapezoid")
    for p in range(0, nc - 1):
        assert abs(np.sum(w * (z - c) ** p)) < 1e-14 * max(1.0, r ** p)
    # p = nc - 1 is the first moment the rule gets wrong (aliasing with 1/(z-c))
    assert abs(np.sum(w * (z - c) ** (nc - 1))) > 1e-3 * r ** (nc - 1)


@pytest.mark.parametrize("rule", ["gl", "trapezoid"])
def test_ellipse_cauchy_integral(rule):
    # (1/2 pi i) oint dz/(z - lam) = 1 inside, 0 outside; many nodes -> near exact
    c, ra, rb = -1.0 + 0.5j, 2.0, 0.5
    z, w = O.quadrature(c, ra, rb, 256, rule)
    f_in = O.filter_function([c + 0.3 + 0.1j, c - 1.0], z, w)
    f_out = O.filter_function([c + 3.0, c + 1.5j], z, w)
    assert np.all(np.abs(f_in - 1.0) < 1e-8)
    assert np.all(np.abs(f_out) < 1e-8)


def test_filter_decays_outside():
    z, w = O.quadrature(0.0, 1.0, 1.0, 8, "gl")
    xs = np.array([1.2, 1.5, 2.0, 4.0, 8.0])
    f = np.abs(O.filter_function(xs, z, w))
    assert np.all(f < 1.0) and np.all(np.diff(f) < 0)
    assert abs(O.filter_function(0.5, z, w)[0] - 1.0) < 1e-3


# ---------------------------------------------------------------- helpers
def test_power_norm_estimate():
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.standard_normal((50, 50)))
    V, _ = np.linalg.qr(rng.standard_normal((50, 50)))
    s = np.linspace(1.0, 5.0, 50)
    s[-1] = 10.0
    A = (U * s) @ V.T
    est = O.power_norm2(A.astype(np.complex128))
    assert est <= 10.0 * (1 + 1e-12)
    assert abs(est - 10.0) < 1e-8
    assert O.power_norm2(None) == 1.0


def test_companion_first_form_eigenvector():
    rng = np.random.default_rng(5)
    m = 4
    Ah = [rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)) for _ in range(3)]
    lam, Y = O.reduced_eig(Ah)
    for i in range(len(lam)):
        P = Ah[0] + lam[i] * Ah[1] + lam[i] ** 2 * Ah[2]
        y = Y[:, i]
        assert np.linalg.norm(P @ y) <= 1e-11 * np.linalg.norm(y) * (1 + abs(lam[i]) ** 2)


def test_brute_force_matches_second_companion():
    for k in (2, 3):
        p = random_pep(20, k, seed=11 + k)
        a = O.brute_force_eigs(p)
        b = second_companion_eigs(problem_mats(p))
        assert match_sets(a, b) < 1e-10


def test_select_ranks_by_normalized_radius():
    lam = np.array([2.0 + 0j, 0.1 + 0.01j, 0.0 + 0.09j, np.inf, 0.5 + 0j])
    # ellipse ra=1, rb=0.1: rho = 2, ~0.141, 0.9, inf, 0.5
    idx = O.select(lam, 0.0, 1.0, 0.1, 3)
    assert list(idx) == [1, 4, 2]


# ---------------------------------------------------------------- Example 1
def test_e1_closed_form_reproduces_table1():
    rows = load_table1(os.path.join(GOLD, "e1_table1.txt"))
    lam = family_eigs(1000, [0.0, 0.0, 1.0], [0.4807, 0.6202, 0.0], 3.0)
    sel = np.sort(lam[(lam.real > -1.6) & (lam.real < -1.5) & (np.abs(lam.imag) < 1e-12)].real)
    assert len(sel) == 20
    assert np.max(np.abs(sel - np.sort([r[1] for r in rows]))) < 6e-11


def test_e1_oracle_reproduces_table1():
    rows = load_table1(os.path.join(GOLD, "e1_table1.txt"))
    p = mass_spring(1000, 0.6202, 0.4807)
    r = O.nlfeast(p, E1_CONTOUR, 22, start_block(1000, 22, 0), tol=1e-10)
    assert r["converged"] and r["iters"] == 3           # "three FEAST iterations"
    lam = np.sort(r["lam"][r["inside"]].real)
    assert len(lam) == 20
    assert np.max(np.abs(lam - np.sort([x[1] for x in rows]))) < 6e-11
    assert np.all(np.abs(r["lam"][r["inside"]].imag) < 1e-12)
    # printed residuals are <= 9.8e-14; FP64 rounding order allows a few times that
    assert np.max(r["abs_res"][r["inside"]]) < 2e-12
    # the two extra Ritz pairs lie outside the interval (Fig. 2 caption)
    assert np.sum(~r["inside"]) == 2


# ---------------------------------------------------------------- closed-form family
@pytest.mark.parametrize("k", [2, 3])
def test_closed_form_family_random(k):
    rng = np.random.default_rng(100 + k)
    n = 60
    c = list(rng.uniform(-1, 1, k + 1))
    d = list(rng.uniform(-1, 1, k + 1))
    c[k], d[k] = 1.0, 0.0                       # monic leading term
    lam_all = family_eigs(n, c, d, 2.5)
    center = lam_all[np.argsort(np.abs(lam_all - np.median(lam_all.real)))[0]]
    dist = np.sort(np.abs(lam_all - center))
    r = 0.5 * (dist[7] + dist[8])               # 8 inside
    p = closed_form_family(n, c, d, 2.5)
    res = O.nlfeast(p, {"center": center, "ra": r, "rb": r, "nc": 16, "rule": "gl"},
                    14, start_block(n, 14, 1), tol=1e-11, maxit=60)
    assert res["converged"]
    got = res["lam"][res["inside"]]
    ref = lam_all[inside_mask(lam_all, center, r, r)]
    assert len(ref) == 8 and len(got) == 8
    assert match_sets(got, ref) < 1e-10
    assert np.all(res["relres"][res["inside"]] <= 1e-11)


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("k", [2, 3])
def test_oracle_matches_qz_random_pep(k):
    n = 40
    p = random_pep(n, k, seed=7 + k)
    lam_all = second_companion_eigs(problem_mats(p))
    lam_all = lam_all[np.isfinite(lam_all)]
    center = np.median(lam_all.real) + 1j * np.median(lam_all.imag)
    dist = np.sort(np.abs(lam_all - center))
    r = 0.5 * (dist[5] + dist[6])               # 6 inside
    res = O.nlfeast(p, {"center": center, "ra": r, "rb": r, "nc": 16, "rule": "gl"},
                    12, start_block(n, 12, 2), tol=1e-11, maxit=80)
    assert res["converged"]
    ref = lam_all[inside_mask(lam_all, center, r, r)]
    got = res["lam"][res["inside"]]
    assert len(got) == len(ref) == 6
    assert match_sets(got, ref) < 1e-10
    assert O.winding_count(p, center, r, r, nsamp=1024) == 6


@pytest.mark.parametrize("k", [2, 3])
def test_shift_invert_nearest_matches_qz(k):
    # the structured shift-invert behind the stored n = 4096 and n = 2048 cubic
    # references, against QZ on the second companion form
    n = 40
    p = random_pep(n, k, seed=11 + k)
    lam_all = second_companion_eigs(problem_mats(p))
    lam_all = lam_all[np.isfinite(lam_all)]
    sigma = 0.31 + 0.17j
    ref = lam_all[np.argsort(np.abs(lam_all - sigma))][:10]
    got = O.shift_invert_nearest(p, sigma, 10)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-12


def test_linear_special_case_matches_eigvals():
    n = 50
    p = linear_problem(n, seed=21)               # T = A - lambda I
    A = p["terms"][0]["A"]
    ev = np.linalg.eigvals(A)
    center = ev[np.argmin(np.abs(ev - 0.2))]
    dist = np.sort(np.abs(ev - center))
    r = 0.5 * (dist[4] + dist[5])
    res = O.nlfeast(p, {"center": center, "ra": r, "rb": r, "nc": 16, "rule": "gl"},
                    10, start_block(n, 10, 4), tol=1e-11, maxit=60)
    assert res["converged"]
    ref = ev[inside_mask(ev, center, r, r)]
    assert match_sets(res["lam"][res["inside"]], ref) < 1e-10


def test_linear_filter_equals_linear_feast():
    # For T(z) = zB - A the Step 4 sum equals sum_j omega_j (z_j B - A)^{-1} B X
    # for ANY X and diagonal Lambda (Sec. 4.2: the integral reduces to the linear one).
    rng = np.random.default_rng(9)
    n, m = 30, 5
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    B = np.eye(n) + 0.1 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    p = {"n": n, "terms": [{"kind": "pow", "p": 0, "scale": -1.0 + 0j, "A": A},
                           {"kind": "pow", "p": 1, "scale": 1.0 + 0j, "A": B}]}
    X = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    lam = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    z, w = O.quadrature(0.1 + 0.2j, 1.3, 0.8, 8, "gl")
    lus = O.factor_nodes(p, z)
    R = O.block_residual(p, X, lam)
    Q = O.filter_update(lus, z, w, X, lam, R)
    Qlin = sum(wj * np.linalg.solve(zj * B - A, B @ X) for zj, wj in zip(z, w))
    assert np.linalg.norm(Q - Qlin) < 1e-11 * np.linalg.norm(Qlin)


def test_block_residual_is_definition():
    p = random_pep(15, 2, seed=3)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((15, 3)) + 0j
    lam = np.array([0.5, -1.0 + 1j, 2j])
    R = O.block_residual(p, X, lam)
    for i in range(3):
        assert np.allclose(R[:, i], O.assemble(p, lam[i]) @ X[:, i], atol=1e-13)


def test_singular_node_detected():
    p = random_pep(10, 2, seed=1)
    z, w = O.quadrature(0.0, 1.0, 1.0, 4, "trapezoid")
    lus = O.factor_nodes(p, z)
    X = np.ones((10, 2), dtype=np.complex128)
    with pytest.raises(O.SingularNode):
        O.filter_update(lus, z, w, X, np.array([z[1], 0.0]), X)


# ---------------------------------------------------------------- planted mistakes
def _small_family_run():
    c, d, a, n = [0.3, -0.2, 1.0], [0.5, 0.4, 0.0], 2.5, 40
    lam_all = family_eigs(n, c, d, a)
    center = lam_all[np.argmin(np.abs(lam_all - (-0.5 + 0.8j)))]
    dist = np.sort(np.abs(lam_all - center))
    r = 0.5 * (dist[5] + dist[6])
    res = O.nlfeast(closed_form_family(n, c, d, a),
                    {"center": center, "ra": r, "rb": r, "nc": 16, "rule": "gl"},
                    10, start_block(n, 10, 5), tol=1e-11, maxit=25)
    ref = lam_all[inside_mask(lam_all, center, r, r)]
    got = res["lam"][res["inside"]]
    ok = res["converged"] and len(got) == len(ref) and match_sets(got, ref) < 1e-10
    return ok


def test_pins_pass_unplanted():
    assert _small_family_run()


@pytest.mark.parametrize("mistake", ["sign_of_solve", "drop_scaling", "conj_weights",
                                     "reversed_coefficients"])
def test_pins_catch_planted_mistake(monkeypatch, mistake):
    """A plausible slip in the filter or the linearisation must fail the pin."""
    import scipy.linalg as sla
    if mistake == "sign_of_solve":
        def bad(lus, z, omega, X, lam, R):
            return sum((X + sla.lu_solve(lu, R)) * (wj / (zj - lam))[None, :]
                       for lu, zj, wj in zip(lus, z, omega))
        monkeypatch.setattr(O, "filter_update", bad)
    elif mistake == "drop_scaling":
        def bad(lus, z, omega, X, lam, R):
            return sum((X - sla.lu_solve(lu, R)) * wj for lu, zj, wj in zip(lus, z, omega))
        monkeypatch.setattr(O, "filter_update", bad)
    elif mistake == "conj_weights":
        good = O.quadrature
        monkeypatch.setattr(O, "quadrature", lambda *a: (good(*a)[0], np.conj(good(*a)[1])))
    elif mistake == "reversed_coefficients":
        good = O.companion
        monkeypatch.setattr(O, "companion", lambda Ahat: good(Ahat[::-1]))
    assert not _small_family_run()


# ---------------------------------------------------------------- stored contours
def test_stored_plain_qep_contour_matches_bruteforce():
    import json
    from workloads import config1_qep
    from tests.closed_forms import second_companion_eigs, problem_mats
    with open(os.path.join(GOLD, "contours.json")) as f:
        w = json.load(f)["qep_plain_n256"]
    p = config1_qep(256, 0)
    lam = second_companion_eigs(problem_mats(p))
    c = complex(*w["center"])
    ins = lam[np.abs(lam - c) < w["ra"]]
    assert len(ins) == w["count"] == 16
    ref = np.array([complex(*x) for x in w["eigs_inside"]])
    assert match_sets(ins, ref) < 1e-11


def _near_singular(problem, lam, steps=2, seed=0):
    """||T(lam) x|| / sum_p |lam|^p ||A_p||_F after inverse iteration from a
    random start (tiny when lam is an eigenvalue)."""
    import scipy.linalg as sla
    mats = problem_mats(problem)
    T = np.zeros_like(mats[0])
    for p in range(len(mats) - 1, -1, -1):
        T = lam * T + mats[p]
    lu = sla.lu_factor(T)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(T.shape[0]) + 1j * rng.standard_normal(T.shape[0])
    for _ in range(steps):
        x = sla.lu_solve(lu, x)
        x /= np.linalg.norm(x)
    scale = sum(abs(lam) ** p * np.linalg.norm(A) for p, A in enumerate(mats))
    return np.linalg.norm(T @ x) / scale


def test_stored_slice_and_mixed_eigenvalues_are_eigenvalues():
    # a sample of the stored references of the 64-disc and mixed-order
    # workloads (from the oracle's shift-invert Arnoldi) checked against T itself
    import json
    from workloads import cubic_pep
    with open(os.path.join(GOLD, "contours.json")) as f:
        g = json.load(f)
    sl = g["slices_n2048"]
    p = cubic_pep(2048, 0)
    picks = [(d, 0) for d in (0, 21, 42, 63) if sl["eigs_inside"][d]]
    for d, i in picks:
        lam = complex(*sl["eigs_inside"][d][i])
        assert abs(lam - complex(*sl["centers"][d])) < sl["r"]
        assert _near_singular(p, lam) < 1e-13
        assert _near_singular(p, lam + 1e-3 * sl["r"]) > 1e-9     # the test can fail
    for q in g["mixed_n"]["problems"]:
        if q["n"] > 1024:
            continue
        pq = cubic_pep(q["n"], q["n"])
        lam = complex(*q["eigs_inside"][3])
        assert _near_singular(pq, lam) < 1e-13
