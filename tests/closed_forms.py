"""Independent references used to pin the oracle (no code shared with it).

* Closed form for A_i = c_i I + d_i S, S = tridiag(-1, a, -1): S has the
  eigenvalues s_j = a - 2 cos(j pi / (n + 1)), and each s_j contributes the k
  roots of the scalar polynomial sum_i (c_i + d_i s_j) lambda^i.
* Brute force through the *second* companion form (block-column form),
  L(lambda) = lambda diag(A_k, I, .., I) + [[A_{k-1}, -I, 0..], [A_{k-2}, 0, -I..],
  .., [A_0, 0, .., 0]], solved by QZ; the oracle uses the first form, so a
  mistake in one linearisation does not hide in the other.
"""
import numpy as np
import scipy.linalg as sla


def tridiag_eigs(n, a):
    j = np.arange(1, n + 1)
    return a - 2.0 * np.cos(j * np.pi / (n + 1))


def family_eigs(n, c, d, a):
    out = []
    for s in tridiag_eigs(n, a):
        coef = [ci + di * s for ci, di in zip(c, d)]      # ascending powers
        out.extend(np.roots(coef[::-1]))
    return np.array(out, dtype=np.complex128)


def second_companion_eigs(mats):
    """mats[p] = coefficient of lambda^p."""
    k = len(mats) - 1
    n = mats[0].shape[0]
    N = k * n
    L0 = np.zeros((N, N), dtype=np.complex128)
    L1 = np.zeros((N, N), dtype=np.complex128)
    for b in range(k):
        L0[b * n:(b + 1) * n, 0:n] = mats[k - 1 - b]
        if b + 1 < k:
            L0[b * n:(b + 1) * n, (b + 1) * n:(b + 2) * n] = -np.eye(n)
            L1[(b + 1) * n:(b + 2) * n, (b + 1) * n:(b + 2) * n] = np.eye(n)
    L1[0:n, 0:n] = mats[k]
    return sla.eigvals(L0, -L1)


def problem_mats(problem):
    n = problem["n"]
    k = max(t["p"] for t in problem["terms"])
    mats = [np.zeros((n, n), dtype=np.complex128) for _ in range(k + 1)]
    for t in problem["terms"]:
        mats[t["p"]] += t["scale"] * (np.eye(n) if t["A"] is None else t["A"])
    return mats


def inside_mask(lam, center, ra, rb):
    d = np.asarray(lam) - center
    with np.errstate(invalid="ignore"):
        return (d.real / ra) ** 2 + (d.imag / rb) ** 2 < 1.0


def match_sets(a, b):
    """Max relative distance of an optimal one-to-one matching of two equal-size sets."""
    from scipy.optimize import linear_sum_assignment
    a = np.asarray(a); b = np.asarray(b)
    assert len(a) == len(b), (len(a), len(b))
    if len(a) == 0:
        return 0.0
    C = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(C)
    return float(np.max(C[r, c] / np.maximum(np.abs(b[c]), 1e-300)))


def load_table1(path):
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            i, lam, res = line.split()
            rows.append((int(i), float(lam), float(res)))
    return rows


def delay_family_eigs(n, c, d, a, tau, branches=range(-3, 4)):
    """Eigenvalues of -lambda I + (c0 I + d0 S) + (c1 I + d1 S) e^{-tau lambda}:
    for each eigenvalue s of S, alpha = c0 + d0 s, beta = c1 + d1 s, the roots of
    -lambda + alpha + beta e^{-tau lambda} = 0 are
    lambda = alpha + W_l(tau beta e^{-tau alpha}) / tau over the Lambert-W branches l."""
    from scipy.special import lambertw
    out = []
    for s in tridiag_eigs(n, a):
        al, be = c[0] + d[0] * s, c[1] + d[1] * s
        for l in branches:
            out.append(al + lambertw(tau * be * np.exp(-tau * al), l) / tau)
    return np.array(out, dtype=np.complex128)
