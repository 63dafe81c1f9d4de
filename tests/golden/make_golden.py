"""Write the golden files of this directory.  Calls only ``oracle/``.

diag_recursion.json -- Algorithm 2 on diagonal data, run by the 50-digit
scalar recursion of ``oracle.diag_mp`` (the special case in which every
iterate stays diagonal; Definition 2).  The float64 oracle, which works
with dense eigen-decompositions, is tested against these values.

Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import math
import os
import sys

import mpmath as mp

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.diag_mp import lowrank_meg_diagonal  # noqa: E402
from oracle.meg import eps_schedule  # noqa: E402


def case_inputs():
    n, r = 12, 3
    lin_c = [math.cos(1.7 * (j + 1)) + 0.05 * j for j in range(n)]
    quad_m = [0.42, 0.27, 0.16, 0.07, 0.04, 0.025, 0.01, 0.005, -0.002, -0.004, 0.0015, -0.001]
    lam0 = [0.5, 0.3, 0.2]
    return n, r, lin_c, quad_m, lam0


def main():
    n, r, lin_c, quad_m, lam0 = case_inputs()
    eps0 = eps_schedule(0)
    # X_1 = (1 - eps_0) X_0 + eps_0/n I with X_0 = diag(lam0) on coordinates 0..r-1
    x1 = [(1 - eps0) * (lam0[j] if j < r else 0.0) + eps0 / n for j in range(n)]
    cases = []
    for name, kind, data, eta in (("linear", "linear", lin_c, 0.7),
                                  ("dense_quadratic", "dense_quadratic", quad_m, 1.0)):
        T = 25
        res = lowrank_meg_diagonal(data, kind, x1, r, T, eta, eps_schedule)
        cases.append({
            "name": name, "kind": kind, "n": n, "r": r, "eta": eta, "T": T,
            "data": data, "lam0": lam0, "eps": {"a": 0.8, "c": 10, "q": 2},
            "x": [[mp.nstr(v, 25) for v in x] for (x, _, _) in res],
            "sig_top": [[mp.nstr(v, 25) for v in s] for (_, s, _) in res],
            "cert": [mp.nstr(c, 25) for (_, _, c) in res],
        })
    with open(os.path.join(HERE, "diag_recursion.json"), "w") as f:
        json.dump({"source": "oracle.diag_mp.lowrank_meg_diagonal, 50 digits; "
                             "Definition 2 / Algorithm 2 on diagonal data",
                   "cases": cases}, f, indent=0)


if __name__ == "__main__":
    main()
