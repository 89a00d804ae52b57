"""Writes tests/golden/rationals.json: RHMC rational coefficients from the
oracle's Remez exchange (oracle/remez.py) and nothing else.

Each entry is the best relative approximation r(x) = a0 + sum a_k/(x + b_k) of
x^p on [lo, hi] of type (d, d) (RHMC, Sec. 2.1 of the paper):
  p = +1/4  pseudofermion heatbath  phi = r(M) R
  p = -1/2  action and force        S_f = phi^dag r(M) phi
for the degrees and ranges of the workloads:
  4^4 trajectory            degree 8 on [1e-3, 64]
  32^3x8 trajectory         degree 15 on [1e-5, 64]
  batched multi-RHS solves  degree 12 on [1e-4, 64]
  small test rationals      degree 6 on [1e-2, 64], degree 4 on [1e-1, 64]

Run from the repository root:  python tests/golden/make_rationals.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import remez  # noqa: E402

CASES = [
    ("d4_1e-1", 4, 1e-1, 64.0),
    ("d6_1e-2", 6, 1e-2, 64.0),
    ("d8_1e-3", 8, 1e-3, 64.0),
    ("d12_1e-4", 12, 1e-4, 64.0),
    ("d15_1e-5", 15, 1e-5, 64.0),
]
POWERS = [("p-1/2", -0.5), ("p+1/4", 0.25)]


def main():
    out = {}
    for name, d, lo, hi in CASES:
        for pname, p in POWERS:
            r = remez.remez(p, lo, hi, d)
            key = "%s_%s" % (pname, name)
            out[key] = dict(power=p, degree=d, lo=lo, hi=hi, a0=r["a0"], a=r["a"], b=r["b"],
                            err=r["err"], spread=r["spread"], iters=r["iters"])
            print(key, "err=%.3e spread=%.1e iters=%d" % (r["err"], r["spread"], r["iters"]),
                  flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rationals.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
