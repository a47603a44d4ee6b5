"""Pins of the oracle's path for non-polynomial T (the delay problem):
closed-form Lambert-W spectra, QZ for the reduced moment solver, the argument
principle, and planted mistakes."""
import numpy as np
import pytest

from oracle import nlfeast_ref as O
from closed_forms import delay_family_eigs, inside_mask, match_sets
from workloads import delay_family, random_pep, start_block

FAM = dict(n=30, c=[-1.0, 0.3], d=[0.5, 0.1], a=2.0, tau=1.0)


def _family_contour():
    lam = delay_family_eigs(FAM["n"], FAM["c"], FAM["d"], FAM["a"], FAM["tau"])
    real0 = np.sort(lam[np.abs(lam.imag) < 1e-12].real)
    center = 0.5 * (real0[10] + real0[3])
    r = 0.5 * (real0[10] - real0[3]) + 1e-3
    return lam, complex(center), float(r)


def test_lambert_w_values_are_eigenvalues():
    """The closed form against the problem's definition: T(lambda) is singular."""
    p = delay_family(**FAM)
    lam = delay_family_eigs(FAM["n"], FAM["c"], FAM["d"], FAM["a"], FAM["tau"])
    for l in lam[::7]:
        smin = np.linalg.svd(O.assemble(p, l), compute_uv=False)[-1]
        assert smin < 1e-12 * max(1.0, abs(l))


def _family_run():
    lam, center, r = _family_contour()
    p = delay_family(**FAM)
    res = O.nlfeast(p, {"center": center, "ra": r, "rb": r, "nc": 16, "rule": "gl"}, 12,
                    start_block(FAM["n"], 12, 3), tol=1e-11, maxit=30)
    ref = lam[inside_mask(lam, center, r, r)]
    got = res["lam"][res["inside"]]
    ok = res["converged"] and len(got) == len(ref) and match_sets(got, ref) < 1e-10
    return ok, res, ref


def test_oracle_delay_family_matches_lambert_w():
    ok, res, ref = _family_run()
    assert ok, (res["converged"], res["iters"], len(ref))
    assert np.all(res["relres"][res["inside"]] <= 1e-11)


def test_delay_count_matches_argument_principle():
    lam, center, r = _family_contour()
    p = delay_family(**FAM)
    assert O.winding_count(p, center, r, r, 512) == int(inside_mask(lam, center, r, r).sum())


def test_beyn_matches_qz_on_a_polynomial():
    """The moment solver alone, on a small polynomial treated as a general T:
    its eigenvalues are those of QZ inside the scaled contour."""
    p = random_pep(12, 2, seed=4)
    G = O.projected_terms(p, np.eye(12, dtype=np.complex128))
    ref_all = O.brute_force_eigs(p)
    center, ra = 0.1 + 0.1j, 0.5
    ref = ref_all[inside_mask(ref_all, center, 1.5 * ra, 1.5 * ra)]
    rng = np.random.default_rng(0)
    V = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    lam, Y = O.reduced_beyn(p, G, center, ra, ra, V)
    assert len(lam) == len(ref) > 0
    assert match_sets(lam, ref) < 1e-8
    lam_n = np.array([O.newton_reduced(p, G, l, Y[:, i])[0] for i, l in enumerate(lam)])
    assert match_sets(lam_n, ref) < 1e-12


@pytest.mark.parametrize("mistake", ["tau_sign", "beyn_first_moment"])
def test_delay_pins_catch_planted_mistake(monkeypatch, mistake):
    if mistake == "tau_sign":
        good = O.f_value
        monkeypatch.setattr(O, "f_value", lambda t, z: good(dict(t, tau=-t["tau"]) if t["kind"] == "exp" else t, z))
    elif mistake == "beyn_first_moment":
        # the second moment replaced by the first: B = U^H A0 W S^-1
        def bad(problem, G, center, ra, rb, probe, nq=256, scale=1.5, rank_tol=1e-12):
            z, w = O.beyn_nodes(center, ra, rb, nq, scale)
            A0 = sum(wk * np.linalg.solve(O.reduced_matrix(problem, G, zk), probe)
                     for zk, wk in zip(z, w))
            U, S, Wh = np.linalg.svd(A0, full_matrices=False)
            r = int(np.sum(S > rank_tol * S[0]))
            Ur, Sr, Wr = U[:, :r], S[:r], Wh[:r, :].conj().T
            lam, Sv = np.linalg.eig((Ur.conj().T @ A0 @ Wr) / Sr[None, :])
            Y = Ur @ Sv
            return lam, Y / np.linalg.norm(Y, axis=0)[None, :]
        monkeypatch.setattr(O, "reduced_beyn", bad)
    ok, _, _ = _family_run()
    assert not ok
