"""Seeded problem generators (coefficient matrices, start blocks).

A problem is a plain dict:

    {"n": int,
     "terms": [{"kind": "pow", "p": int, "scale": complex, "A": ndarray | None}, ...
               {"kind": "exp", "tau": float, "scale": complex, "A": ndarray | None}],
     "name": str}

meaning T(lambda) = sum_t scale_t * f_t(lambda) * A_t with f = lambda**p ("pow")
or f = exp(-tau*lambda) ("exp"), and A_t = None standing for the identity
(the problem statement T(lambda)x = 0 of Sec. 2, Eq. for the matrix polynomial
P(lambda) = sum_i lambda^i A_i).  Matrices are complex128, C order.

Random draws use numpy's PCG64 ``default_rng(seed)``.  Nothing here computes
eigenvalues, contours or any step of the method.
"""
import numpy as np

__all__ = [
    "tridiag", "sym_gauss", "complex_gauss", "start_block",
    "mass_spring", "closed_form_family", "config1_qep", "config2_qep",
    "random_pep", "linear_problem", "delay_problem", "cubic_pep", "delay_family",
    "serving_requests",
]


def tridiag(n, diag, off):
    """Dense n x n tridiagonal matrix with constant diagonal and off-diagonal."""
    T = np.zeros((n, n), dtype=np.complex128)
    idx = np.arange(n)
    T[idx, idx] = diag
    T[idx[:-1], idx[:-1] + 1] = off
    T[idx[1:], idx[1:] - 1] = off
    return T


def sym_gauss(rng, n):
    """Dense symmetric N(0,1)/sqrt(n): (G + G^T)/sqrt(2)/sqrt(n), G real Gaussian."""
    G = rng.standard_normal((n, n))
    return ((G + G.T) / np.sqrt(2.0) / np.sqrt(n)).astype(np.complex128)


def complex_gauss(rng, n, m=None):
    """Dense complex N(0,1)/sqrt(n): (G1 + i G2)/sqrt(2)/sqrt(n), real plane first."""
    m = n if m is None else m
    G1 = rng.standard_normal((n, m))
    G2 = rng.standard_normal((n, m))
    return (G1 + 1j * G2) / np.sqrt(2.0) / np.sqrt(n)


def start_block(n, m0, seed):
    """Initial subspace X0 (n x m0): complex standard normal (N + iN)/sqrt(2),
    drawn from default_rng(seed) as the real plane then the imaginary plane."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((n, m0))
    im = rng.standard_normal((n, m0))
    return np.ascontiguousarray((re + 1j * im) / np.sqrt(2.0))


def _pow_terms(mats):
    return [{"kind": "pow", "p": p, "scale": 1.0 + 0j, "A": A} for p, A in enumerate(mats)]


def mass_spring(n, tau, kappa):
    """Mass-spring quadratic problem of Example 1/2 (Sec. 5):
    A2 = I, A1 = tau*S, A0 = kappa*S with S = tridiag(-1, 3, -1)."""
    S = tridiag(n, 3.0, -1.0)
    terms = [{"kind": "pow", "p": 0, "scale": 1.0 + 0j, "A": kappa * S},
             {"kind": "pow", "p": 1, "scale": 1.0 + 0j, "A": tau * S},
             {"kind": "pow", "p": 2, "scale": 1.0 + 0j, "A": None}]
    return {"n": n, "terms": terms, "name": f"mass_spring_n{n}"}


def closed_form_family(n, c, d, a):
    """A_i = c_i I + d_i S with S = tridiag(-1, a, -1) (every A_i commutes with S)."""
    S = tridiag(n, a, -1.0)
    I = np.eye(n, dtype=np.complex128)
    mats = [ci * I + di * S for ci, di in zip(c, d)]
    return {"n": n, "terms": _pow_terms(mats), "name": f"closed_form_n{n}"}


def config1_qep(n=256, seed=0):
    """Quadratic lambda^2 I + lambda A1 + A0 with A0 = tridiag(-1,2,-1) + 0.01 S1,
    A1 = 0.05 I + 0.02 S2; S1 then S2 drawn as dense symmetric N(0,1)/sqrt(n)."""
    rng = np.random.default_rng(seed)
    S1 = sym_gauss(rng, n)
    S2 = sym_gauss(rng, n)
    A0 = tridiag(n, 2.0, -1.0) + 0.01 * S1
    A1 = 0.05 * np.eye(n, dtype=np.complex128) + 0.02 * S2
    terms = [{"kind": "pow", "p": 0, "scale": 1.0 + 0j, "A": A0},
             {"kind": "pow", "p": 1, "scale": 1.0 + 0j, "A": A1},
             {"kind": "pow", "p": 2, "scale": 1.0 + 0j, "A": None}]
    return {"n": n, "terms": terms, "name": f"qep_plain_n{n}"}


def config2_qep(n=4096, seed=0):
    """Quadratic lambda^2 M + lambda C + K:
    M = I + 0.1 diag(U[0,1]); C = 0.02 G/sqrt(n) (real, non-symmetric);
    K = Qo diag(linspace(0.1, 100, n)) Qo^T, Qo from the QR of a real Gaussian with
    the signs of diag(R) folded in.  Draw order: U, then G_C, then G_Q."""
    rng = np.random.default_rng(seed)
    u = rng.random(n)
    GC = rng.standard_normal((n, n))
    GQ = rng.standard_normal((n, n))
    M = np.diag(1.0 + 0.1 * u).astype(np.complex128)
    C = (0.02 / np.sqrt(n)) * GC
    Qo, Ro = np.linalg.qr(GQ)
    Qo = Qo * np.sign(np.diag(Ro))[None, :]
    K = (Qo * np.linspace(0.1, 100.0, n)[None, :]) @ Qo.T
    K = 0.5 * (K + K.T)
    terms = [{"kind": "pow", "p": 0, "scale": 1.0 + 0j, "A": K.astype(np.complex128)},
             {"kind": "pow", "p": 1, "scale": 1.0 + 0j, "A": C.astype(np.complex128)},
             {"kind": "pow", "p": 2, "scale": 1.0 + 0j, "A": M}]
    return {"n": n, "terms": terms, "name": f"qep_mixed_n{n}"}


def random_pep(n, k, seed):
    """Dense complex N(0,1)/sqrt(n) coefficients A_0..A_k."""
    rng = np.random.default_rng(seed)
    mats = [complex_gauss(rng, n) for _ in range(k + 1)]
    return {"n": n, "terms": _pow_terms(mats), "name": f"random_pep_n{n}_k{k}"}


def cubic_pep(n, seed):
    return random_pep(n, 3, seed)


def linear_problem(n, seed, B=None):
    """T(lambda) = A - lambda B (B = identity when None): the standard or
    generalized linear problem written as a degree-1 matrix polynomial."""
    rng = np.random.default_rng(seed)
    A = complex_gauss(rng, n)
    terms = [{"kind": "pow", "p": 0, "scale": 1.0 + 0j, "A": A},
             {"kind": "pow", "p": 1, "scale": -1.0 + 0j, "A": B}]
    return {"n": n, "terms": terms, "name": f"linear_n{n}"}


def delay_problem(n, seed, tau=1.0):
    """T(lambda) = -lambda I + A0 + A1 exp(-tau lambda):
    A0 = G1/sqrt(n) - 2I, A1 = 0.5 G2/sqrt(n) (real Gaussians, G1 then G2)."""
    rng = np.random.default_rng(seed)
    G1 = rng.standard_normal((n, n))
    G2 = rng.standard_normal((n, n))
    A0 = (G1 / np.sqrt(n) - 2.0 * np.eye(n)).astype(np.complex128)
    A1 = (0.5 * G2 / np.sqrt(n)).astype(np.complex128)
    terms = [{"kind": "pow", "p": 1, "scale": -1.0 + 0j, "A": None},
             {"kind": "pow", "p": 0, "scale": 1.0 + 0j, "A": A0},
             {"kind": "exp", "tau": float(tau), "scale": 1.0 + 0j, "A": A1}]
    return {"n": n, "terms": terms, "name": f"delay_n{n}"}


def delay_family(n, c, d, a, tau=1.0):
    """T(lambda) = -lambda I + (c0 I + d0 S) + (c1 I + d1 S) exp(-tau lambda),
    S = tridiag(-1, a, -1): every eigenvalue is alpha + W_l(tau beta e^{-tau alpha})/tau
    for an eigenvalue s of S (alpha = c0 + d0 s, beta = c1 + d1 s) and a branch l
    of the Lambert W function."""
    S = tridiag(n, a, -1.0)
    I = np.eye(n, dtype=np.complex128)
    terms = [{"kind": "pow", "p": 1, "scale": -1.0 + 0j, "A": None},
             {"kind": "pow", "p": 0, "scale": 1.0 + 0j, "A": c[0] * I + d[0] * S},
             {"kind": "exp", "tau": float(tau), "scale": 1.0 + 0j, "A": c[1] * I + d[1] * S}]
    return {"n": n, "terms": terms, "name": f"delay_family_n{n}"}


def serving_requests(num, seed=2024, rate=200.0, n_lo=128, n_hi=4096):
    """A seeded stream of solve requests: Poisson arrivals at `rate` per second
    (exponential gaps), n log-uniform in [n_lo, n_hi], degree 2 or 3 with
    dense complex N(0,1)/sqrt(n) coefficients (``random_pep(n, k, coef_seed)``),
    8 to 16 quadrature nodes, a wanted eigenvalue count in [4, 64] and a
    random point of the spectral bulk (modulus in [0.6, 1.5], uniform angle)
    about which the contour is drawn.  Only random draws: the circle itself
    (radius, count, enclosed eigenvalues) is computed elsewhere."""
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for q in range(num):
        t += rng.exponential(1.0 / rate)
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        k = int(rng.choice([2, 3]))
        nc = int(rng.integers(8, 17))
        want = int(rng.integers(4, 65))
        rho, th = rng.uniform(0.6, 1.5), rng.uniform(0.0, 2.0 * np.pi)
        out.append({"t": float(t), "n": n, "k": k, "coef_seed": 7000 + q, "nc": nc,
                    "want": want, "point": complex(rho * np.cos(th), rho * np.sin(th))})
    return out
