"""Writes tests/golden/contours.json: the contour of each benchmark workload and
the eigenvalues it encloses, computed ONLY with the oracle's brute-force tools
(QZ on the companion pencil for n = 256, shift-invert Arnoldi for n = 4096).

Run from the repository root:  python tests/golden/make_contours.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import brute_force_eigs, shift_invert_nearest, winding_count  # noqa: E402
from workloads import config1_qep, config2_qep  # noqa: E402


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


def main():
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
    with open(os.path.join(ROOT, "tests", "golden", "contours.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
