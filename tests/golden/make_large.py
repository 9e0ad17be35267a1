"""Write tests/golden/large_samples.json: FP64 oracle values, computed one by
one, for the two large single instances 12x12 D=2 (seed 1212) and 8x8 D=3
(seed 883).  The whole observable set would take the row-sweep oracle hours
(8x8 D=3: 248 row absorptions of ~1.5e11 multiply-adds each), so each sample
is one expectation value with only two cached boundaries
(oracle.expect_one): the norm, a site <X_k>, and <Z_i Z_j> on bonds inside a
corner and across both cuts of the quadrant partition the library chooses
for energies ((6, 6) at 12x12, (4, 4) at 8x8).

It calls nothing but ``oracle`` and the seeded input generator, so every
stored value is the oracle's (Sec. 3, Eqs. norm, mx, cij; Sec. 4 row order).
Run from the repository root:  python tests/golden/make_large.py
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1908_08553_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "large_samples.json")

# (L, W, D, seed, [(op, site i, site j, what)])  sites are r * W + c
CASES = [
    (12, 12, 2, 1212, [("x", 7 * 12 + 3, 0, "site (7,3)"),
                       ("zz", 2 * 12 + 5, 2 * 12 + 6, "horizontal bond across the vertical cut"),
                       ("zz", 5 * 12 + 9, 6 * 12 + 9, "vertical bond across the horizontal cut"),
                       ("zz", 9 * 12 + 2, 9 * 12 + 3, "horizontal bond inside a corner"),
                       ("zz", 1 * 12 + 1, 2 * 12 + 1, "vertical bond inside a corner")]),
    (8, 8, 3, 883, [("x", 2 * 8 + 5, 0, "site (2,5)"),
                    ("zz", 1 * 8 + 3, 1 * 8 + 4, "horizontal bond across the vertical cut"),
                    ("zz", 3 * 8 + 6, 4 * 8 + 6, "vertical bond across the horizontal cut")]),
]


def main():
    out = {"cite": "FP64 row-sweep oracle (Sec. 4 row scheme) of Eqs. norm, mx and cij (Sec. 3), one "
                   "expectation value per call; inputs: seeded uniform[-1,1) site tensors",
           "cases": []}
    for L, W, D, seed, samples in CASES:
        A = inputs.random_lattice(L, W, D, seed)
        case = {"L": L, "W": W, "D": D, "seed": seed, "samples": []}
        for op, i, j, what in samples:
            t0 = time.time()
            v, nm, ne = oracle.expect_one(L, W, D, A, op, i, j)
            case["samples"].append({"op": op, "i": i, "j": j, "what": what, "value": v,
                                    "norm_mant": nm, "norm_exp2": ne, "seconds": round(time.time() - t0, 1)})
            print(f"{L}x{W} D={D} {op} {i} {j}: {v!r} ({time.time() - t0:.0f} s)", flush=True)
        case["oracle_threads"] = oracle.num_threads()
        out["cases"].append(case)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
