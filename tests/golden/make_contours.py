"""Writes tests/golden/contours.json: the contour of each benchmark workload and
the eigenvalues it encloses, computed ONLY with the oracle (QZ on the companion
pencil for n = 256, shift-invert Arnoldi for n = 4096 and for the 64 discs of
the n = 2048 cubic, an oracle solve plus an argument-principle count for the
n = 2048 delay problem).

Run from the repository root:  python tests/golden/make_contours.py
(`python tests/golden/make_contours.py delay_n2048` or `... slices_n2048`
refreshes that entry only.)
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import (assemble, brute_force_eigs, nlfeast, normalized_radius,  # noqa: E402
                    shift_invert_nearest, winding_count)
from workloads import (config1_qep, config2_qep, cubic_pep, delay_problem, random_pep,  # noqa: E402
                       serving_requests, start_block)


def circle_around(lam, target, count):
    """Center = eigenvalue nearest `target` rounded to 3 decimals; radius = midpoint
    of the count-th and (count+1)-th distances from that center."""
    c0 = lam[np.argmin(np.abs(lam - target))]
    center = complex(round(c0.real, 3), round(c0.imag, 3))
    d = np.sort(np.abs(lam - center))
    r = 0.5 * (d[count - 1] + d[count])
    gap = (d[count] - d[count - 1]) / r
    inside = lam[np.abs(lam - center) < r]
    return center, float(r), float(gap), inside


def adaptive_winding(problem, center, ra, rb, nsamp=512, tol=np.pi / 4, depth=10):
    """Argument-principle count with the samples refined (bisection in theta)
    wherever arg det T changes by more than `tol` between neighbours."""
    def phase(th):
        z = center + ra * np.cos(th) + 1j * rb * np.sin(th)
        sign, _ = np.linalg.slogdet(assemble(problem, z))
        return np.angle(sign)

    def span(ta, pa, tb, pb, d):
        dp = np.angle(np.exp(1j * (pb - pa)))
        if abs(dp) <= tol or d == 0:
            return dp
        tm = 0.5 * (ta + tb)
        pm = phase(tm)
        return span(ta, pa, tm, pm, d - 1) + span(tm, pm, tb, pb, d - 1)

    th = 2.0 * np.pi * np.arange(nsamp + 1) / nsamp
    ph = [phase(t) for t in th[:-1]]
    ph.append(ph[0])
    total = sum(span(th[i], ph[i], th[i + 1], ph[i + 1], depth) for i in range(nsamp))
    return int(round(total / (2.0 * np.pi)))


def delay_contour():
    """C3: n = 2048 delay problem, ellipse with axes 2:1 at -0.9 (the rightmost
    cluster), semi-axis chosen at a gap of the normalised radii of the
    eigenvalues an oracle solve finds on a larger ellipse."""
    n = 2048
    p = delay_problem(n, 0)
    c = -0.9 + 0j
    big = nlfeast(p, {"center": c, "ra": 0.2, "rb": 0.1, "nc": 24, "rule": "gl"}, 72,
                  start_block(n, 72, 0), tol=1e-11, maxit=40)
    assert big["converged"]
    lam = big["lam"][big["inside"]]
    rho = 0.2 * normalized_radius(lam, c, 0.2, 0.1)       # in units of ra
    rs = np.sort(rho)
    count = 29                                             # largest relative gap near 32
    ra = 0.5 * (rs[count - 1] + rs[count])
    gap = (rs[count] - rs[count - 1]) / ra
    inside = lam[rho < ra]
    assert len(inside) == count
    w = adaptive_winding(p, c, ra, ra / 2)
    assert w == count, (w, count)
    return p, c, float(ra), float(gap), inside, w


def main():
    path = os.path.join(ROOT, "tests", "golden", "contours.json")
    if sys.argv[1:] == ["delay_n2048"]:          # refresh that entry only
        main_delay_only(path)
        return
    if sys.argv[1:] == ["slices_n2048"]:
        main_slices_only(path)
        return
    if sys.argv[1:] == ["mixed_n"]:
        main_mixed_only(path)
        return
    if sys.argv[1:2] == ["serving"]:
        main_serving(int(sys.argv[2]) if len(sys.argv) > 2 else SERVING_REQUESTS)
        return
    out = {}
    p1 = config1_qep(256, 0)
    lam1 = brute_force_eigs(p1)
    lam1 = lam1[np.isfinite(lam1)]
    c1, r1, g1, in1 = circle_around(lam1, 1.0j, 16)
    w1 = winding_count(p1, c1, r1, r1, nsamp=2048)
    assert w1 == 16 == len(in1), (w1, len(in1))
    out["qep_plain_n256"] = {
        "generator": "config1_qep(n=256, seed=0)", "center": [c1.real, c1.imag],
        "ra": r1, "rb": r1, "nc": 8, "rule": "gl", "m0": 24, "count": 16,
        "relative_gap": g1, "winding_count": w1,
        "eigs_inside": [[x.real, x.imag] for x in sorted(in1, key=lambda v: (v.real, v.imag))],
        "method": "QZ on the 512 x 512 first companion pencil"}
    print("C1", c1, r1, g1)

    p2 = config2_qep(4096, 0)
    target = 1j * np.sqrt(50.0)
    near = shift_invert_nearest(p2, target, 48)
    c0 = near[0]
    center = complex(round(c0.real, 3), round(c0.imag, 3))
    lam2 = shift_invert_nearest(p2, center, 110)
    c2, r2, g2, in2 = circle_around(lam2, center, 64)
    assert len(in2) == 64
    out["qep_mixed_n4096"] = {
        "generator": "config2_qep(n=4096, seed=0)", "center": [c2.real, c2.imag],
        "ra": r2, "rb": r2, "nc": 16, "rule": "gl", "m0": 96, "count": 64,
        "relative_gap": g2,
        "eigs_inside": [[x.real, x.imag] for x in sorted(in2, key=lambda v: (v.real, v.imag))],
        "method": "shift-invert Arnoldi (110 nearest) on the 8192 first companion pencil"}
    print("C2", c2, r2, g2)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    main_delay_only(path)
    main_slices_only(path)
    main_mixed_only(path)


def main_delay_only(path):
    with open(path) as f:
        out = json.load(f)
    _, c3, r3, g3, in3, w3 = delay_contour()
    out["delay_n2048"] = {
        "generator": "delay_problem(n=2048, seed=0, tau=1)", "center": [c3.real, c3.imag],
        "ra": r3, "rb": r3 / 2, "nc": 24, "rule": "gl", "m0": 48, "count": len(in3),
        "relative_gap": g3, "winding_count": w3,
        "eigs_inside": [[x.real, x.imag] for x in sorted(in3, key=lambda v: (v.real, v.imag))],
        "method": "oracle solve on the ellipse (0.2, 0.1) with m0 = 72 to 1e-11; "
                  "count checked by the argument principle with adaptive sampling"}
    print("C3", c3, r3, g3, w3)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


# spectrum slicing: the square of side 0.8 centred at 0.5 + 0.25i cut into an
# 8 x 8 grid of cells, one inscribed disc (radius 0.05) per cell
SLICE_CENTER, SLICE_SIDE, SLICE_GRID = 0.5 + 0.25j, 0.8, 8


def slice_discs():
    step = SLICE_SIDE / SLICE_GRID
    x0 = SLICE_CENTER.real - SLICE_SIDE / 2 + step / 2
    y0 = SLICE_CENTER.imag - SLICE_SIDE / 2 + step / 2
    centers = [complex(x0 + i * step, y0 + j * step)
               for j in range(SLICE_GRID) for i in range(SLICE_GRID)]
    return centers, step / 2


def main_slices_only(path):
    """Every eigenvalue in each disc, from the 24 nearest its center (shift-invert
    Arnoldi on the 6144 x 6144 companion pencil); the 24th must lie outside, so
    none is missed, and no disc may hold 12 or more."""
    with open(path) as f:
        out = json.load(f)
    p = cubic_pep(2048, 0)
    centers, r = slice_discs()
    eigs, margin = [], np.inf
    for c in centers:
        near = shift_invert_nearest(p, c, 24)
        d = np.abs(near - c) / r
        assert d[-1] > 1.0, (c, d[-1])
        inside = near[d < 1.0]
        assert len(inside) < 12, (c, len(inside))
        margin = min(margin, float(np.min(np.abs(d - 1.0))))
        eigs.append([[x.real, x.imag] for x in sorted(inside, key=lambda v: (v.real, v.imag))])
    out["slices_n2048"] = {
        "generator": "cubic_pep(n=2048, seed=0)",
        "centers": [[c.real, c.imag] for c in centers], "r": r, "nc": 8, "rule": "gl", "m0": 16,
        "count": int(sum(len(e) for e in eigs)), "counts": [len(e) for e in eigs],
        "min_boundary_margin": margin, "eigs_inside": eigs,
        "method": "shift-invert Arnoldi (24 nearest each disc center) on the first companion "
                  "pencil through one n x n LU per disc"}
    print("C4", len(centers), "discs,", out["slices_n2048"]["count"], "eigenvalues, margin", margin)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


# mixed-order batch: one cubic with complex Gaussian coefficients per order
MIXED_ORDERS = (256, 512, 1024, 2048, 4096)


def main_mixed_only(path):
    """Per order n: the circle around the eigenvalue nearest 0.5 + 0.25i (rounded
    to 3 decimals) holding 8 eigenvalues (radius in the gap after the 8th
    nearest), and those 8, from the 24 nearest by shift-invert Arnoldi."""
    with open(path) as f:
        out = json.load(f)
    probs = []
    for n in MIXED_ORDERS:
        p = cubic_pep(n, n)
        near = shift_invert_nearest(p, 0.5 + 0.25j, 24)
        c0 = near[0]
        center = complex(round(c0.real, 3), round(c0.imag, 3))
        lam = shift_invert_nearest(p, center, 24)
        d = np.sort(np.abs(lam - center))
        r = 0.5 * (d[7] + d[8])
        gap = (d[8] - d[7]) / r
        inside = lam[np.abs(lam - center) < r]
        assert len(inside) == 8 and d[-1] > r
        probs.append({"n": n, "generator": f"cubic_pep(n={n}, seed={n})",
                      "center": [center.real, center.imag], "r": float(r), "relative_gap": float(gap),
                      "eigs_inside": [[x.real, x.imag] for x in sorted(inside, key=lambda v: (v.real, v.imag))]})
        print("mixed", n, center, r, gap)
    out["mixed_n"] = {"problems": probs, "nc": 8, "rule": "gl", "m0": 16, "count": 8 * len(probs),
                      "method": "shift-invert Arnoldi (24 nearest the center) on the first companion "
                                "pencil through one n x n LU"}
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


# serving stream (random PEPs of mixed n and degree): its own file
SERVING_REQUESTS = 104          # 8 warm-up + 96 timed requests


def serving_circle(q):
    """One request of ``serving_requests``: the eigenvalues nearest its random
    point (shift-invert Arnoldi, want + 12 of them); the count is taken in
    [want - 3, want + 3] (clipped to [4, 64]) at the widest relative gap of
    the sorted distances, the radius in the middle of that gap."""
    import os as _os
    _os.environ.setdefault("OMP_NUM_THREADS", "2")
    p = random_pep(q["n"], q["k"], q["coef_seed"])
    c = q["point"]
    lam = shift_invert_nearest(p, c, q["want"] + 12)
    d = np.sort(np.abs(lam - c))
    lo, hi = max(4, q["want"] - 3), min(64, q["want"] + 3)
    kk = max(range(lo, hi + 1), key=lambda j: (d[j] - d[j - 1]) / d[j])
    r = 0.5 * (d[kk - 1] + d[kk])
    inside = lam[np.abs(lam - c) < r]
    assert len(inside) == kk and d[-1] > r
    return {"t": q["t"], "n": q["n"], "k": q["k"], "coef_seed": q["coef_seed"], "nc": q["nc"],
            "center": [c.real, c.imag], "r": float(r), "count": int(kk),
            "m0": int(np.ceil(1.5 * kk)), "relative_gap": float((d[kk] - d[kk - 1]) / r),
            "eigs_inside": [[x.real, x.imag] for x in sorted(inside, key=lambda v: (v.real, v.imag))]}


def main_serving(num):
    """tests/golden/serving_stream.json: the circles and enclosed eigenvalues of
    the first `num` requests of ``serving_requests()`` (oracle only)."""
    import multiprocessing as mp
    reqs = serving_requests(num)
    with mp.get_context("spawn").Pool(4) as pool:
        rows = pool.map(serving_circle, reqs, chunksize=1)
    out = {"generator": "serving_requests(num=%d, seed=2024, rate=200)" % num,
           "coefficients": "random_pep(n, k, coef_seed)", "rule": "gl",
           "method": "shift-invert Arnoldi (want + 12 nearest the random point) on the first "
                     "companion pencil through one n x n LU",
           "requests": rows}
    with open(os.path.join(ROOT, "tests", "golden", "serving_stream.json"), "w") as f:
        json.dump(out, f, indent=0)
    print("serving", num, "requests,", sum(r["count"] for r in rows), "eigenvalues")


if __name__ == "__main__":
    main()
