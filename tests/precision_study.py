"""How precise must the node solves of Algorithm 1 be?  A CPU study.

Sec. 4.2 relates NLFEAST to residual inverse iteration: Step 4 solves
T(z_j) Y_j = T(X, Lambda), and the right-hand side is the block residual,
which tends to zero as X converges.  An error of relative size eps in the
solve therefore perturbs Q by eps times something that vanishes with the
residual, so a low-precision node factorisation should slow the convergence
(by a factor near 1 + eps kappa(T(z_j))) without limiting the accuracy reached,
as long as Steps 1-3 stay in FP64.  The paper does not quantify this; this
module measures it by running the FP64 oracle with emulated node solves:

  fp64    LAPACK complex128 (the oracle's own solve);
  fp32    LAPACK complex64 factorisation and triangular solves;
  tf32    blocked right-looking LU in complex64: FP32 panels with partial
          pivoting, and every trailing update (and every off-diagonal block
          product of the two triangular solves) with both operands rounded to
          TF32 (10-bit significand, round to nearest even) and FP32 sums;
  tf32x3  the same with each operand split x = hi + lo, hi = tf32(x),
          lo = tf32(x - hi), and the three products hi hi + hi lo + lo hi;

each with 0, 1 or 2 refinement sweeps Y <- Y + LU^{-1}(R - T(z_j) Y), whose
residual is formed in FP64.  The right-hand side enters the low-precision
solves rounded to complex64 and the solution returns as complex128.

    python tests/precision_study.py --modes fp64,tf32 --sweeps 0,1
        # n = 4096 QEP, 16 nodes, m0 = 96: ~1 to 40 minutes per (mode, sweeps)
        # on 8 cores (the emulated TF32 factorisations and FP64 sweeps dominate)
    python tests/precision_study.py --workload qep_plain_n256     # seconds

Test infrastructure: this file calls the oracle and numpy only.
"""
import argparse
import json
import os
import sys
import time

import numpy as np
import scipy.linalg as sla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle.nlfeast_ref as O  # noqa: E402
import workloads  # noqa: E402

MODES = ("fp64", "fp32", "tf32x3", "tf32")
PANEL = 64


def tf32(x):
    """Round a float32 array to TF32 (1 sign, 8 exponent, 10 significand bits),
    to nearest with ties to even; finite inputs only."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    lsb = (u >> np.uint32(13)) & np.uint32(1)
    r = (u + np.uint32(0x0FFF) + lsb) & np.uint32(0xFFFFE000)
    return r.view(np.float32)


def tf32c(z):
    """TF32 rounding of the real and imaginary planes of a complex64 array."""
    out = np.empty(z.shape, dtype=np.complex64)
    out.real = tf32(z.real)
    out.imag = tf32(z.imag)
    return out


def split(a, mode):
    """The operand pieces a mode multiplies with: (a,), (tf32(a),) or
    (hi, lo) with hi = tf32(a), lo = tf32(a - hi)."""
    if mode == "tf32":
        return (tf32c(a),)
    if mode == "tf32x3":
        hi = tf32c(a)
        return (hi, tf32c(a - hi))
    return (a,)


def product(a, b, mode):
    """a @ b in complex64 with FP32 sums; a given as ``split(a, mode)``, b as is."""
    if mode == "tf32":
        return a[0] @ tf32c(b)
    if mode == "tf32x3":
        ah, al = a
        bh = tf32c(b)
        bl = tf32c(b - bh)
        return ah @ bh + (ah @ bl + al @ bh)
    return a[0] @ b


class BlockedLU:
    """Right-looking LU with partial pivoting, column panels of PANEL, of a
    complex64 matrix; the trailing updates use ``product(.., mode)``.  The
    off-diagonal blocks of the factors are split once for the solves."""

    def __init__(self, A, mode):
        A = np.array(A, dtype=np.complex64, order="C")
        n = A.shape[0]
        perm = np.arange(n)
        for k in range(0, n, PANEL):
            e = min(k + PANEL, n)
            lu, piv = sla.lu_factor(A[k:, k:e], check_finite=False)
            A[k:, k:e] = lu
            for i, p in enumerate(piv):              # the panel's interchanges, whole rows
                if p != i:
                    a, b = k + i, k + p
                    A[[a, b], :k] = A[[b, a], :k]
                    A[[a, b], e:] = A[[b, a], e:]
                    perm[[a, b]] = perm[[b, a]]
            if e < n:
                A[k:e, e:] = sla.solve_triangular(A[k:e, k:e], A[k:e, e:], lower=True,
                                                  unit_diagonal=True, check_finite=False)
                A[e:, e:] -= product(split(A[e:, k:e], mode), A[k:e, e:], mode)
        self.A, self.perm, self.mode, self.n = A, perm, mode, n
        blocks = range(0, n, PANEL)
        self.L = {k: split(A[k + PANEL:, k:k + PANEL], mode) for k in blocks if k + PANEL < n}
        self.U = {k: split(A[:k, k:k + PANEL], mode) for k in blocks if k > 0}

    def solve(self, B):
        """T^{-1} B (B complex64, n x m): P, then L, then U by blocks."""
        A, mode, n = self.A, self.mode, self.n
        Y = np.array(B[self.perm], dtype=np.complex64)
        for k in range(0, n, PANEL):
            e = min(k + PANEL, n)
            Y[k:e] = sla.solve_triangular(A[k:e, k:e], Y[k:e], lower=True,
                                          unit_diagonal=True, check_finite=False)
            if e < n:
                Y[e:] -= product(self.L[k], Y[k:e], mode)
        for k in reversed(range(0, n, PANEL)):
            e = min(k + PANEL, n)
            Y[k:e] = sla.solve_triangular(A[k:e, k:e], Y[k:e], lower=False,
                                          check_finite=False)
            if k > 0:
                Y[:k] -= product(self.U[k], Y[k:e], mode)
        return Y


def node_solvers(problem, z, mode, sweeps):
    """One callable R -> T(z_j)^{-1} R per node, at the given precision, with
    `sweeps` refinement sweeps whose residual is formed in FP64."""
    solvers = []
    for zj in z:
        T = O.assemble(problem, zj)
        if mode == "fp64":
            f = sla.lu_factor(T)
            low = lambda R, f=f: sla.lu_solve(f, R)
        elif mode == "fp32":
            f = sla.lu_factor(T.astype(np.complex64))
            low = lambda R, f=f: sla.lu_solve(f, R.astype(np.complex64)).astype(np.complex128)
        else:
            f = BlockedLU(T, mode)
            low = lambda R, f=f: f.solve(R.astype(np.complex64)).astype(np.complex128)
        if sweeps == 0:
            solvers.append(low)
            continue

        def refined(R, low=low, zj=zj):
            Y = low(R)
            for _ in range(sweeps):
                Y = Y + low(R - O.assemble(problem, zj) @ Y)
            return Y
        solvers.append(refined)
    return solvers


def run(problem, contour, m0, X0, mode, sweeps, tol, maxit, norms):
    """One solve; also returns the (Ritz values, relative residuals) of every
    Step 3, recorded around the oracle's residual function."""
    z, _ = O.quadrature(complex(contour["center"]), contour["ra"], contour["rb"],
                        contour["nc"], contour["rule"])
    t0 = time.perf_counter()
    lus = node_solvers(problem, z, mode, sweeps)
    t1 = time.perf_counter()
    trace, plain = [], O.relative_residuals

    def recorded(problem_, R, lam, norms_):
        rr = plain(problem_, R, lam, norms_)
        trace.append((np.array(lam), np.array(rr)))
        return rr
    O.relative_residuals = recorded
    try:
        r = O.nlfeast(problem, contour, m0, X0, tol=tol, maxit=maxit, lus=lus, norms=norms)
    finally:
        O.relative_residuals = plain
    t2 = time.perf_counter()
    r["trace"] = trace
    return r, t1 - t0, t2 - t1


def found(trace, ref, tol=1e-10):
    """Per iteration: how many reference eigenvalues have a Ritz pair with
    relative residual <= tol whose eigenvalue lies within tol (relative)."""
    out = []
    for lam, rr in trace:
        good = lam[rr <= tol]
        out.append(int(sum(1 for e in ref if good.size and np.min(np.abs(good - e)) <= tol * abs(e))))
    return out


def study(workload="qep_mixed_n4096", modes=MODES, sweeps=(0, 1, 2), tol=1e-10, maxit=40,
          seed=0, log=print):
    """Every (mode, sweeps) run of one stored workload from the same start block;
    eigenvalues compared with the FP64 run's (the first mode must be fp64)."""
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "contours.json")))[workload]
    gen, kw = gold["generator"].split("(", 1)
    args = dict(a.split("=") for a in kw.rstrip(")").replace(" ", "").split(","))
    problem = getattr(workloads, gen)(**{k: int(v) for k, v in args.items()})
    contour = {"center": complex(*gold["center"]), "ra": gold["ra"], "rb": gold["rb"],
               "nc": gold["nc"], "rule": gold["rule"]}
    m0, n = gold["m0"], problem["n"]
    eigs = np.array([complex(*e) for e in gold["eigs_inside"]])
    X0 = workloads.start_block(n, m0, seed)
    norms = O.term_norms(problem)
    rows, ref = [], None
    for mode in modes:
        for s in (sweeps if mode != "fp64" else (0,)):
            r, tf, ts = run(problem, contour, m0, X0, mode, s, tol, maxit, norms)
            lam = r["lam"][r["inside"]]
            if ref is None:
                ref = lam
            err = max((min(abs(ref - l)) / abs(l) for l in lam), default=0.0)
            fnd = found(r["trace"], eigs, tol)
            all_found = next((i + 1 for i, f in enumerate(fnd) if f == len(eigs)), None)
            row = {"mode": mode, "sweeps": s, "iters": r["iters"], "converged": r["converged"],
                   "iters_all_true_pairs": all_found, "found": fnd,
                   "inside": int(r["inside"].sum()), "max_relres": float(r["relres"][r["inside"]].max()),
                   "max_rel_eig_err_vs_fp64": float(err),
                   "history": [float(h) for h in r["history"]],
                   "factor_s": round(tf, 1), "solve_s": round(ts, 1)}
            rows.append(row)
            log(json.dumps(row))
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="qep_mixed_n4096",
                    choices=["qep_mixed_n4096", "qep_plain_n256"])
    ap.add_argument("--maxit", type=int, default=40)
    ap.add_argument("--modes", default=",".join(MODES),
                    help="comma-separated; the first must be fp64 (the reference run)")
    ap.add_argument("--sweeps", default="0,1,2")
    ap.add_argument("--out", default=None, help="write the rows as JSON here")
    a = ap.parse_args()
    rows = study(a.workload, modes=a.modes.split(","),
                 sweeps=tuple(int(x) for x in a.sweeps.split(",")), maxit=a.maxit)
    print("| node solves | refinement sweeps | iterations (Step 3 test) | iterations until every "
          "reference pair is found | inside | max relres | max eigenvalue error vs FP64 |")
    print("|---|---|---|---|---|---|---|")
    for r in rows:
        print(f"| {r['mode']} | {r['sweeps']} | {r['iters']} | {r['iters_all_true_pairs']} | "
              f"{r['inside']} | {r['max_relres']:.1e} | {r['max_rel_eig_err_vs_fp64']:.1e} |")
    if a.out:
        json.dump(rows, open(a.out, "w"), indent=1)


if __name__ == "__main__":
    main()
