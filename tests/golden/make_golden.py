"""Writes the stored expected values under tests/golden/ by calling only the
oracle (oracle/closed_forms.py, oracle/rule.py).  Run from the repository
root:  python tests/golden/make_golden.py

* paper_integrands.json: the paper's fixed-parameter test integrands f1..f5
  (Sec. 4.1, equations for f1..f5) mapped onto the five families, with their
  closed-form integrals over [0,1]^n.
* rule_weights.json: the degree-9 rule's generators (squared radii) and
  orbit counts, the basic weights as exact fractions, and the four null rules
  at 40 significant digits, for n = 2..8.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import closed_forms as cf  # noqa: E402
from oracle import rule  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def paper_integrands():
    cases = []
    # f1 = cos(sum_i i x_i), n = 8 (Sec. 4.1, Eq. for f1): oscillatory, u = 0, a_i = i
    cases.append(("f1", cf.OSCILLATORY, 8, [0.0] + [float(i) for i in range(1, 9)]))
    # f2 = prod_i (1/50^2 + (x_i - 1/2)^2)^-1, n = 6 (Eq. for f2): product peak, c = 50, w = 1/2
    cases.append(("f2", cf.PRODUCT_PEAK, 6, [50.0] * 6 + [0.5] * 6))
    # f3 = (1 + sum_i i x_i)^(-n-1), n = 3 and 8 (Eq. for f3): corner peak, a_i = i
    for n in (3, 8):
        cases.append((f"f3_d{n}", cf.CORNER_PEAK, n, [float(i) for i in range(1, n + 1)]))
    # f4 = exp(-625 sum (x_i - 1/2)^2), n = 5 and 8 (Eq. for f4): Gaussian, a = 25, w = 1/2
    for n in (5, 8):
        cases.append((f"f4_d{n}", cf.GAUSSIAN, n, [25.0] * n + [0.5] * n))
    # f5 = exp(-10 sum |x_i - 1/2|), n = 5 and 8 (Eq. for f5): C0, a = 10, w = 1/2
    for n in (5, 8):
        cases.append((f"f5_d{n}", cf.C0, n, [10.0] * n + [0.5] * n))
    # f6 = exp(sum_i (i + 4) x_i) if x_i < (3 + i)/10, n = 6 (Eq. for f6): discontinuous family
    cases.append(("f6", cf.DISCONTINUOUS, 6, [float(i + 4) for i in range(1, 7)] + [(3 + i) / 10 for i in range(1, 7)]))
    # f7 = (sum x_i^2)^11, n = 8 (Eq. for f7): box power, exact rational
    cases.append(("f7_d8", cf.BOX_POWER, 8, [11.0]))
    out = {"_source": "paper Sec. 4.1 (test integrands f1..f7; f8 has no closed form); values from "
                      "oracle/closed_forms.py",
           "cases": []}
    for name, fam, n, p in cases:
        out["cases"].append({"name": name, "family": fam, "dim": n, "params": p,
                             "integral": repr(cf.closed_form(fam, n, p))})
    return out


def rule_weights():
    out = {"_source": "degree-9 fully symmetric rule (paper Sec. 2.1, Sec. 3.2; generators and null rules "
                      "as read in oracle/rule.py), computed by oracle/rule.py", "rules": {}}
    for n in range(2, 9):
        gens, cnt, w, _, nulls = rule.exact_rule(n)
        out["rules"][str(n)] = {
            "generators_lambda": [[str(x) for x in g] for g in gens],
            "counts": cnt,
            "basic": [str(x) for x in w],
            "null": [[format(x, ".40e") for x in u] for u in nulls],
        }
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "paper_integrands.json"), "w") as f:
        json.dump(paper_integrands(), f, indent=1)
    with open(os.path.join(HERE, "rule_weights.json"), "w") as f:
        json.dump(rule_weights(), f, indent=1)
    print("written")
