"""Plain FP64 CPU oracle of nonlinear FEAST (NLFEAST).

Gavin, Miedlar, Polizzi, "FEAST Eigensolver for Nonlinear Eigenvalue Problems"
(arXiv 1801.09794).  Every function names the passage it follows.

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` (to check the GPU result) and by ``bench.py``'s
CPU-baseline / reference leg.  The GPU library never imports, links or calls
it, and it shares no code with the GPU library: both consume only the seeded
problems of ``workloads/``.

Everything is complex128 / float64 on the host, written for readability and
not for speed: numpy/scipy LAPACK routines (LU, QR, QZ) serve as single steps.

Readings of points the paper leaves open:

* Quadrature (Algorithm 1 inputs; Step 4): the contour is
  z(theta) = c + ra*cos(theta) + i*rb*sin(theta), theta in [0, 2*pi)
  (a circle when ra == rb), and omega_j = w_j * z'(theta_j) / (2*pi*i),
  i.e. the 1/(2*pi*i) factor of the integral is folded into the weights.
  Default rule: Gauss-Legendre with n_c points on [0, 2*pi].
* Step 4's right factor (z_j I - Lambda)^{-1} is diagonal, so it scales
  column i by 1/(z_j - lambda_i).
* Step 2 "closest to the interior of C": rank by the normalised radius
  rho(lambda) = |((Re(lambda - c))/ra, (Im(lambda - c))/rb)|_2, with a
  stable sort on (rho, Re lambda, Im lambda); inside means rho < 1.
* Step 3's test is the relative residual
  ||T(lambda_i) x_i||_2 / sum_t |scale_t f_t(lambda_i)| * ||A_t||_2 with
  ||x_i||_2 = 1, over the Ritz values strictly inside C, where ||A_t||_2 is
  estimated by 30 power iterations on A^H A from the normalised all-ones
  vector (identity: 1).  The iteration count counts executions of Step 1,
  and the test is not taken before one filter application.
* Step 1 for polynomial T: the projected matrix polynomial is linearised in
  the first companion form (Sec. 2, the k = 2 pencil there, generalised to
  degree k) and solved by QZ; the Ritz vector is the last block of the pencil
  eigenvector.
* Step 1 for non-polynomial T (the paper names no reduced solver): the
  projected problem That(z) = sum_t scale_t f_t(z) Q^H A_t Q is solved by the
  first two contour moments of That^{-1} (Beyn's method, which the paper
  cites among the contour methods; here it is only the m0 x m0 reduced
  solver): trapezoid rule with 256 nodes on the contour scaled by 1.5 about
  its centre, an m0 x m0 seeded complex-normal probe, rank by
  sigma > 1e-12 sigma_1; then at most 5 Newton steps (inverse iteration for
  nonlinear problems) per pair.  Slots the moments leave empty are filled with
  lambda = c + 1.5 ra (outside C, never tested) and unit coordinate vectors.
"""
import numpy as np
import scipy.linalg as sla

__all__ = [
    "quadrature", "filter_function", "f_value", "assemble", "power_norm2",
    "term_norms", "projected_coefficients", "companion", "reduced_eig",
    "normalized_radius", "select", "ritz_vectors", "block_residual",
    "relative_residuals", "filter_update", "orthonormalize", "factor_nodes",
    "nlfeast", "brute_force_eigs", "winding_count", "shift_invert_nearest",
    "SingularNode", "f_derivative", "projected_terms", "reduced_matrix", "beyn_nodes",
    "reduced_beyn", "newton_reduced", "reduced_solve_general",
]


class SingularNode(ArithmeticError):
    """A Ritz value coincides with a quadrature node (Step 4 divides by z_j - lambda_i)."""


# --------------------------------------------------------------------------
# Contour and quadrature (Algorithm 1, inputs; Step 4)
# --------------------------------------------------------------------------
def quadrature(center, ra, rb, nc, rule="gl"):
    """Nodes z_j and weights omega_j with sum_j omega_j g(z_j) ~ (1/(2 pi i)) oint g(z) dz.

    Algorithm 1 takes "a set of n_c quadrature nodes and weights"; Step 4 sums
    omega_j * (...) * (z_j I - Lambda)^{-1}.  The parametrisation and the rule are
    the readings stated in the module docstring.
    """
    if nc < 1:
        raise ValueError("nc must be positive")
    if rule == "gl":
        x, w = np.polynomial.legendre.leggauss(nc)
        theta = np.pi * (x + 1.0)
        wt = np.pi * w
    elif rule == "trapezoid":
        theta = 2.0 * np.pi * (np.arange(nc) + 0.5) / nc
        wt = np.full(nc, 2.0 * np.pi / nc)
    elif rule == "gl_halves":
        if nc % 2:
            raise ValueError("gl_halves needs an even nc")
        x, w = np.polynomial.legendre.leggauss(nc // 2)
        t0 = 0.5 * np.pi * (x + 1.0)
        theta = np.concatenate([t0, t0 + np.pi])
        wt = np.concatenate([0.5 * np.pi * w, 0.5 * np.pi * w])
    else:
        raise ValueError(f"unknown rule {rule!r}")
    z = center + ra * np.cos(theta) + 1j * rb * np.sin(theta)
    dz = -ra * np.sin(theta) + 1j * rb * np.cos(theta)
    omega = wt * dz / (2j * np.pi)
    return z.astype(np.complex128), omega.astype(np.complex128)


def filter_function(lam, z, omega):
    """Scalar filter f(lambda) = sum_j omega_j / (z_j - lambda): the coefficient of
    x_i in column i of Step 4 (it approximates 1 inside C and 0 outside)."""
    lam = np.atleast_1d(np.asarray(lam, dtype=np.complex128))
    return (omega[None, :] / (z[None, :] - lam[:, None])).sum(axis=1)


# --------------------------------------------------------------------------
# The matrix function T (Sec. 2: T(lambda) = sum_i lambda^i A_i; Sec. 6 for
# non-polynomial f)
# --------------------------------------------------------------------------
def f_value(term, z):
    """Scalar function of one term: lambda**p or exp(-tau*lambda), times its scale."""
    z = np.asarray(z, dtype=np.complex128)
    if term["kind"] == "pow":
        v = z ** term["p"]
    elif term["kind"] == "exp":
        v = np.exp(-term["tau"] * z)
    else:
        raise ValueError(term["kind"])
    return term["scale"] * v


def f_derivative(term, z):
    """d/dz of f_value: scale * p z^(p-1), or scale * (-tau) exp(-tau z)."""
    z = np.asarray(z, dtype=np.complex128)
    if term["kind"] == "pow":
        p = term["p"]
        v = p * z ** (p - 1) if p > 0 else np.zeros_like(z)
    elif term["kind"] == "exp":
        v = -term["tau"] * np.exp(-term["tau"] * z)
    else:
        raise ValueError(term["kind"])
    return term["scale"] * v


def assemble(problem, z):
    """T(z) = sum_t scale_t f_t(z) A_t as a dense matrix (A_t None = identity)."""
    n = problem["n"]
    T = np.zeros((n, n), dtype=np.complex128)
    for t in problem["terms"]:
        c = complex(f_value(t, z))
        if t["A"] is None:
            T[np.diag_indices(n)] += c
        else:
            T += c * t["A"]
    return T


def power_norm2(A, iters=30):
    """||A||_2 estimated by `iters` power steps on A^H A from ones/sqrt(n)."""
    if A is None:
        return 1.0
    n = A.shape[1]
    v = np.full(n, 1.0 / np.sqrt(n), dtype=np.complex128)
    s = 0.0
    for _ in range(iters):
        w = A.conj().T @ (A @ v)
        s = np.linalg.norm(w)
        if s == 0.0:
            return 0.0
        v = w / s
    return float(np.sqrt(s))


def term_norms(problem, iters=30):
    return np.array([power_norm2(t["A"], iters) for t in problem["terms"]])


# --------------------------------------------------------------------------
# Step 1: projected problem Q^H T(lambda) Q y = 0, solved by linearisation
# --------------------------------------------------------------------------
def projected_coefficients(problem, Q):
    """Ahat_p = sum_{t: f_t = lambda^p} scale_t Q^H A_t Q, p = 0..k (Step 1)."""
    k = max(t["p"] for t in problem["terms"] if t["kind"] == "pow")
    m = Q.shape[1]
    Ahat = [np.zeros((m, m), dtype=np.complex128) for _ in range(k + 1)]
    for t in problem["terms"]:
        if t["kind"] != "pow":
            raise NotImplementedError("projected_coefficients is for polynomial T")
        AQ = Q if t["A"] is None else t["A"] @ Q
        Ahat[t["p"]] += t["scale"] * (Q.conj().T @ AQ)
    return Ahat


def companion(Ahat):
    """First companion form L(lambda) = L0 + lambda*L1 of sum_p lambda^p Ahat_p.

    Sec. 2 writes it for k = 2 as lambda*[[A2, 0], [0, I]] + [[A1, A0], [-I, 0]]
    with eigenvectors [lambda x; x]; for degree k the first block row holds
    A_{k-1} .. A_0, the sub-diagonal blocks are -I, and L1 = diag(A_k, I, .., I).
    The eigenvector is [lambda^{k-1} y; ...; lambda y; y].
    """
    k = len(Ahat) - 1
    m = Ahat[0].shape[0]
    N = k * m
    L0 = np.zeros((N, N), dtype=np.complex128)
    L1 = np.zeros((N, N), dtype=np.complex128)
    for b in range(k):
        L0[0:m, b * m:(b + 1) * m] = Ahat[k - 1 - b]
    for b in range(1, k):
        L0[b * m:(b + 1) * m, (b - 1) * m:b * m] = -np.eye(m)
        L1[b * m:(b + 1) * m, b * m:(b + 1) * m] = np.eye(m)
    L1[0:m, 0:m] = Ahat[k]
    return L0, L1


def reduced_eig(Ahat):
    """All eigenpairs of the projected polynomial (Step 1) by QZ on the companion.

    Returns eigenvalues (k*m,) and the vectors y (m, k*m) taken from the last
    block of each pencil eigenvector.
    """
    L0, L1 = companion(Ahat)
    m = Ahat[0].shape[0]
    lam, Z = sla.eig(L0, -L1)
    return lam, Z[-m:, :]


# --------------------------------------------------------------------------
# Step 1 for non-polynomial T (reading in the module docstring)
# --------------------------------------------------------------------------
def projected_terms(problem, Q):
    """G_t = Q^H A_t Q for every term (A_t None: Q^H Q), so that the projected
    problem is That(z) = sum_t scale_t f_t(z) G_t (Step 1 for any T)."""
    out = []
    for t in problem["terms"]:
        AQ = Q if t["A"] is None else t["A"] @ Q
        out.append(Q.conj().T @ AQ)
    return out


def reduced_matrix(problem, G, z, derivative=False):
    """That(z) (or That'(z)) = sum_t scale_t f_t(z) G_t."""
    f = f_derivative if derivative else f_value
    M = np.zeros_like(G[0])
    for t, Gt in zip(problem["terms"], G):
        M = M + complex(f(t, z)) * Gt
    return M


def beyn_nodes(center, ra, rb, nq=256, scale=1.5):
    """Trapezoid nodes on the ellipse scaled by `scale` about `center`, with the
    1/(2 pi i) and dz/dtheta folded into the weights: sum_k w_k g(z_k)
    approximates (1/(2 pi i)) closed-integral g(z) dz."""
    theta = 2.0 * np.pi * (np.arange(nq) + 0.5) / nq
    a, b = scale * ra, scale * rb
    z = center + a * np.cos(theta) + 1j * b * np.sin(theta)
    dz = -a * np.sin(theta) + 1j * b * np.cos(theta)
    w = dz * (2.0 * np.pi / nq) / (2j * np.pi)
    return z, w


def reduced_beyn(problem, G, center, ra, rb, probe, nq=256, scale=1.5, rank_tol=1e-12):
    """Beyn's moments A0 = sum_k w_k That(z_k)^{-1} V, A1 = sum_k w_k z_k That(z_k)^{-1} V;
    A0 = U S W^H, rank r by S > rank_tol S_1; B = U_r^H A1 W_r S_r^{-1}; the
    eigenvalues of B are the eigenvalues of That inside the scaled contour, with
    vectors U_r s (unit)."""
    z, w = beyn_nodes(center, ra, rb, nq, scale)
    m = G[0].shape[0]
    A0 = np.zeros((m, probe.shape[1]), dtype=np.complex128)
    A1 = np.zeros_like(A0)
    for zk, wk in zip(z, w):
        Y = np.linalg.solve(reduced_matrix(problem, G, zk), probe)
        A0 += wk * Y
        A1 += (wk * zk) * Y
    U, S, Wh = np.linalg.svd(A0, full_matrices=False)
    r = int(np.sum(S > rank_tol * S[0])) if S.size and S[0] > 0 else 0
    if r == 0:
        return np.zeros(0, dtype=np.complex128), np.zeros((m, 0), dtype=np.complex128)
    Ur, Sr, Wr = U[:, :r], S[:r], Wh[:r, :].conj().T
    B = (Ur.conj().T @ A1 @ Wr) / Sr[None, :]
    lam, Sv = np.linalg.eig(B)
    Y = Ur @ Sv
    return lam, Y / np.linalg.norm(Y, axis=0)[None, :]


def newton_reduced(problem, G, lam, y, steps=5):
    """Newton's method on [That(l) y = 0, y^H y = 1] (inverse iteration for
    nonlinear problems): u = That(l)^{-1} That'(l) y, l <- l - 1/(y^H u),
    y <- u / |u|; at most `steps` steps, stopping at FP64 rounding."""
    y = y / np.linalg.norm(y)
    for _ in range(steps):
        try:
            u = np.linalg.solve(reduced_matrix(problem, G, lam),
                                reduced_matrix(problem, G, lam, derivative=True) @ y)
        except np.linalg.LinAlgError:     # an exact eigenvalue already
            break
        yu = np.vdot(y, u)
        if yu == 0 or not np.isfinite(yu):
            break
        dl = -1.0 / yu
        lam = lam + dl
        y = u / np.linalg.norm(u)
        if abs(dl) <= 4.0 * np.finfo(float).eps * max(abs(lam), 1.0):
            break
    return lam, y


def reduced_solve_general(problem, G, center, ra, rb, m0, probe):
    """Steps 1-2 for any T: Beyn's eigenpairs of That inside the 1.5x contour,
    polished by Newton, ranked by (rho, Re, Im); at most m0 kept; the empty
    slots get lambda = c + 1.5 ra (outside C) and unit coordinate vectors."""
    lam_b, Y_b = reduced_beyn(problem, G, center, ra, rb, probe)
    m = G[0].shape[0]
    lam = []
    Y = []
    for i in range(lam_b.size):
        l, y = newton_reduced(problem, G, lam_b[i], Y_b[:, i])
        lam.append(l)
        Y.append(y)
    lam = np.array(lam, dtype=np.complex128)
    Y = np.array(Y, dtype=np.complex128).T.reshape(m, -1)
    if lam.size:
        order = select(lam, center, ra, rb, min(m0, lam.size))
        lam, Y = lam[order], Y[:, order]
    nf = m0 - lam.size
    if nf > 0:
        fill_l = np.full(nf, center + 1.5 * ra, dtype=np.complex128)
        fill_y = np.zeros((m, nf), dtype=np.complex128)
        for q in range(nf):
            fill_y[(lam.size + q) % m, q] = 1.0
        lam = np.concatenate([lam, fill_l])
        Y = np.concatenate([Y, fill_y], axis=1)
    return lam, Y


def normalized_radius(lam, center, ra, rb):
    """rho(lambda) of the Step 2 reading; rho < 1 means inside C."""
    lam = np.asarray(lam, dtype=np.complex128)
    d = lam - center
    with np.errstate(invalid="ignore", over="ignore"):
        rho = np.sqrt((d.real / ra) ** 2 + (d.imag / rb) ** 2)
    rho = np.where(np.isfinite(rho), rho, np.inf)
    return rho


def select(lam, center, ra, rb, m0):
    """Step 2: indices of the m0 Ritz values closest to the interior of C."""
    rho = normalized_radius(lam, center, ra, rb)
    re = np.where(np.isfinite(lam.real), lam.real, np.inf)
    im = np.where(np.isfinite(lam.imag), lam.imag, np.inf)
    order = np.lexsort((im, re, rho))
    return order[:m0]


def ritz_vectors(Q, Y):
    """X = Q Y with unit columns (Step 2)."""
    X = Q @ Y
    return X / np.linalg.norm(X, axis=0)[None, :]


# --------------------------------------------------------------------------
# Step 3: block residual and its test
# --------------------------------------------------------------------------
def block_residual(problem, X, lam):
    """T(X, Lambda) = sum_t A_t X diag(scale_t f_t(lambda_i)) (Sec. 4.2, the block
    residual function; for a polynomial sum_i A_i X Lambda^i)."""
    R = np.zeros_like(X)
    for t in problem["terms"]:
        fx = f_value(t, lam)
        AX = X if t["A"] is None else t["A"] @ X
        R += AX * fx[None, :]
    return R


def relative_residuals(problem, R, lam, norms):
    """||r_i||_2 / sum_t |scale_t f_t(lambda_i)| ||A_t||_2 (the Step 3 reading)."""
    den = np.zeros(len(lam))
    for t, nt in zip(problem["terms"], norms):
        den += np.abs(f_value(t, lam)) * nt
    return np.linalg.norm(R, axis=0) / den


# --------------------------------------------------------------------------
# Step 4: the contour-quadrature filter
# --------------------------------------------------------------------------
def factor_nodes(problem, z):
    """LU factors of T(z_j) for every node (fixed shifts, so done once per contour)."""
    return [sla.lu_factor(assemble(problem, zj)) for zj in z]


def filter_update(lus, z, omega, X, lam, R):
    """Step 4: Q = sum_j omega_j (X - T(z_j)^{-1} T(X, Lambda)) (z_j I - Lambda)^{-1}.

    lus[j] is either T(z_j)'s LU factors (scipy's ``lu_factor`` pair) or a
    callable R -> T(z_j)^{-1} R; the callable form lets a test substitute an
    inexact solve (Sec. 4.2 reads the filter as residual inverse iteration,
    which tolerates one)."""
    Q = np.zeros_like(X)
    for lu, zj, wj in zip(lus, z, omega):
        d = zj - lam
        if np.any(d == 0):
            raise SingularNode("Ritz value on a quadrature node")
        Yj = lu(R) if callable(lu) else sla.lu_solve(lu, R)
        Q += (X - Yj) * (wj / d)[None, :]
    return Q


def orthonormalize(Q):
    """Steps 0 and 5: orthonormal basis of span(Q) by Householder QR."""
    q, _ = np.linalg.qr(Q, mode="reduced")
    return q


# --------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------
def nlfeast(problem, contour, m0, X0, tol=1e-10, maxit=50, lus=None, norms=None, probe_seed=12345):
    """Algorithm 1 (NLFEAST for T(lambda)x = 0); polynomial T through the
    companion linearisation, any other T through the Beyn reduced solver
    (probe drawn from `probe_seed`).

    contour: {"center": complex, "ra": float, "rb": float, "nc": int, "rule": str}.
    Returns a dict with the m0 selected Ritz values ``lam`` and unit vectors ``X``,
    their relative residuals ``relres``, the ``inside`` mask, the iteration count
    ``iters`` (executions of Step 1), ``converged`` and the per-iteration maximum
    relative residual over the inside pairs ``history``.
    """
    c, ra, rb = complex(contour["center"]), float(contour["ra"]), float(contour["rb"])
    z, omega = quadrature(c, ra, rb, int(contour["nc"]), contour.get("rule", "gl"))
    if lus is None:
        lus = factor_nodes(problem, z)
    if norms is None:
        norms = term_norms(problem)
    Q = orthonormalize(np.asarray(X0, dtype=np.complex128))          # Step 0
    history = []
    converged = False
    it = 0
    polynomial = all(t["kind"] == "pow" for t in problem["terms"])
    probe = None
    if not polynomial:
        rng = np.random.default_rng(probe_seed)
        probe = (rng.standard_normal((m0, m0)) + 1j * rng.standard_normal((m0, m0))) / np.sqrt(2.0)
    for it in range(1, maxit + 1):
        if polynomial:
            Ahat = projected_coefficients(problem, Q)                  # Step 1
            lam_all, Y_all = reduced_eig(Ahat)
            sel = select(lam_all, c, ra, rb, m0)                       # Step 2
            lam = lam_all[sel]
            X = ritz_vectors(Q, Y_all[:, sel])
        else:
            G = projected_terms(problem, Q)                            # Steps 1-2
            lam, Y = reduced_solve_general(problem, G, c, ra, rb, m0, probe)
            X = ritz_vectors(Q, Y)
        R = block_residual(problem, X, lam)                            # Step 3
        rr = relative_residuals(problem, R, lam, norms)
        ins = normalized_radius(lam, c, ra, rb) < 1.0
        history.append(float(rr[ins].max()) if ins.any() else 0.0)
        if it > 1 and np.all(rr[ins] <= tol):
            converged = True
            break
        if it == maxit:
            break
        Q = orthonormalize(filter_update(lus, z, omega, X, lam, R))    # Steps 4, 5
    return {"lam": lam, "X": X, "relres": rr, "inside": ins, "iters": it,
            "converged": converged, "history": history, "norms": norms,
            "abs_res": np.linalg.norm(R, axis=0)}


# --------------------------------------------------------------------------
# Brute-force references used to pin the oracle and to build test contours
# --------------------------------------------------------------------------
def _power_matrices(problem):
    n = problem["n"]
    k = max(t["p"] for t in problem["terms"])
    mats = [np.zeros((n, n), dtype=np.complex128) for _ in range(k + 1)]
    for t in problem["terms"]:
        if t["kind"] != "pow":
            raise NotImplementedError
        mats[t["p"]] += t["scale"] * (np.eye(n) if t["A"] is None else t["A"])
    return mats


def brute_force_eigs(problem):
    """Every eigenvalue of a small polynomial problem: QZ on the full companion."""
    L0, L1 = companion(_power_matrices(problem))
    return sla.eigvals(L0, -L1)


def winding_count(problem, center, ra, rb, nsamp=2048):
    """Number of eigenvalues inside C by the argument principle:
    (1/2 pi) * total change of arg det T(z) along C, with det T from an LU."""
    theta = 2.0 * np.pi * np.arange(nsamp + 1) / nsamp
    zs = center + ra * np.cos(theta) + 1j * rb * np.sin(theta)
    ph = np.empty(nsamp + 1)
    for s, zz in enumerate(zs):
        sign, _ = np.linalg.slogdet(assemble(problem, zz))
        ph[s] = np.angle(sign)
    return int(round((np.unwrap(ph)[-1] - ph[0]) / (2.0 * np.pi)))


def shift_invert_nearest(problem, sigma, nev):
    """The nev eigenvalues of a polynomial problem nearest sigma, by shift-invert
    Arnoldi on the first companion pencil L(lambda) = L0 + lambda L1 (`companion`),
    eigenvalue theta = 1/(sigma - lambda) of (L0 + sigma L1)^{-1} L1.  Block
    elimination of the companion structure reduces each application to one solve
    with P(sigma) (one n x n LU, no k n x k n factorisation): for b = L1 v
    (b_0 = A_k v_0, b_j = v_j) and c_{k-1} = 0, c_j = b_{j+1} + sigma c_{j+1},
        P(sigma) u_{k-1} = b_0 + sigma A_k c_0 + sum_j A_{k-1-j} c_j,
        u_j = sigma u_{j+1} - b_{j+1}  (j = k-2 .. 0)."""
    from scipy.sparse.linalg import LinearOperator, eigs
    mats = _power_matrices(problem)
    k = len(mats) - 1
    n = problem["n"]
    Ps = mats[k].copy()
    for p in range(k - 1, -1, -1):
        Ps = sigma * Ps + mats[p]
    lu = sla.lu_factor(Ps)

    def op(v):
        v = np.asarray(v).reshape(k, n)
        b = [mats[k] @ v[0]] + [v[j] for j in range(1, k)]
        c = [None] * k
        c[k - 1] = np.zeros(n, dtype=np.complex128)
        for j in range(k - 2, -1, -1):
            c[j] = b[j + 1] + sigma * c[j + 1]
        rhs = b[0] + sigma * (mats[k] @ c[0])
        for j in range(k):
            rhs = rhs + mats[k - 1 - j] @ c[j]
        u = [None] * k
        u[k - 1] = sla.lu_solve(lu, rhs)
        for j in range(k - 2, -1, -1):
            u[j] = sigma * u[j + 1] - b[j + 1]
        return np.concatenate(u)

    L = LinearOperator((k * n, k * n), matvec=op, dtype=np.complex128)
    theta = eigs(L, k=nev, which="LM", return_eigenvectors=False, tol=1e-13,
                 ncv=min(k * n, max(2 * nev + 1, 160)))
    lam = sigma - 1.0 / theta
    return lam[np.argsort(np.abs(lam - sigma))]
