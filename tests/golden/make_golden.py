"""Writes the closed-form fixtures in this folder.  Uses only the Python `math` module.

gll_nodes.json  -- Gauss-Lobatto-Legendre nodes on [0, 1] for p = 1..4 from their closed
                   forms on [-1, 1]: p = 3 interior t = +-1/sqrt(5); p = 4 interior
                   t = 0, +-sqrt(3/7); mapped by x = (1 + t)/2 (node family of the Q_p
                   elements, Section 2.2).
piola_diag.json -- first Piola stress of Eq. hypref at F = diag(a, b, c):
                   P_ii = mu (F_ii - 1/F_ii) + 2 lambda ln(abc) / F_ii, off-diagonal zero.
"""
import json
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def gll():
    s5 = 1.0 / math.sqrt(5.0)
    s37 = math.sqrt(3.0 / 7.0)
    to01 = lambda ts: [(1.0 + t) / 2.0 for t in ts]
    return {
        "1": to01([-1.0, 1.0]),
        "2": to01([-1.0, 0.0, 1.0]),
        "3": to01([-1.0, -s5, s5, 1.0]),
        "4": to01([-1.0, -s37, 0.0, s37, 1.0]),
    }


def piola_cases():
    out = []
    for mu, lam, F in [(1.0, 1.5, (1.1, 0.9, 1.05)), (0.4225, 0.6338, (0.95, 1.0, 1.2)),
                       (1.0, 49.0, (1.0, 1.0, 0.97))]:
        lnJ = math.log(F[0] * F[1] * F[2])
        out.append({"mu": mu, "lam": lam, "F": list(F),
                    "P_diag": [mu * (x - 1.0 / x) + 2.0 * lam * lnJ / x for x in F]})
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "gll_nodes.json"), "w") as f:
        json.dump({"source": __doc__.strip(), "nodes": gll()}, f, indent=1)
    with open(os.path.join(HERE, "piola_diag.json"), "w") as f:
        json.dump({"source": __doc__.strip(), "cases": piola_cases()}, f, indent=1)
