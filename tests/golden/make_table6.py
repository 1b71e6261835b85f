"""Writes table6_flops.json: the formulas of Table 6 (FLOPs of the operations of
Alg. 1 and of one epoch, with n points, block size b and l right-hand sides)
evaluated at the bench workload (n = 262,144, b = 4096, l = 16) and at the
n = 4096 RBF case (b = 512, l = 1).  The formulas are the paper's; the script
only evaluates them.  Run from the repository root:

    python tests/golden/make_table6.py
"""
import json
import os

ROWS = {
    "cache_cholesky": ("n b^2 / 3", lambda n, b, l: n * b * b / 3),
    "gs_rule": ("2 n l", lambda n, b, l: 2 * n * l),
    "weight_update": ("(b^2 + b) l", lambda n, b, l: (b * b + b) * l),
    "residual_update": ("(b^2 + 2 n b + n) l", lambda n, b, l: (b * b + 2 * n * b + n) * l),
    "epoch_total": ("((2 + 3 / b) n^2 + (2 b + 1) n) l", lambda n, b, l: ((2 + 3 / b) * n * n + (2 * b + 1) * n) * l),
}
CASES = [("matern52_ard (bench)", 262144, 4096, 16), ("small_rbf", 4096, 512, 1)]


def table() -> dict:
    cases = []
    for name, n, b, l in CASES:
        c = {"name": name, "n": n, "b": b, "l": l}
        for key, (_, f) in ROWS.items():
            c[key] = f(n, b, l)
        cases.append(c)
    return {"source": "Table 6 (FLOP counting in Alg. 1, appendix 'FLOPs in Alg. 1'): per-operation FLOPs with n "
                      "points, block size b and l right-hand sides; no hidden constant in the leading terms",
            "rows": {k: v[0] for k, v in ROWS.items()}, "cases": cases}


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "table6_flops.json")
    with open(out, "w") as f:
        json.dump(table(), f, indent=1)
        f.write("\n")
    print("wrote", out)
