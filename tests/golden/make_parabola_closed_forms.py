"""Writes parabola_closed_forms.txt: Eq. 4 and Eq. 5 (Sec. II.C) at delta = mu
in closed form, with Python's math module alone (no oracle, no engine).

At u = (delta - mu) / sigma = 0 the sigmoid's exp(-u^2/2) is 1 and
1 -/+ erf(0) is 1, so Eq. 4's second term vanishes and
w = c1 / (pi ln2 sigma^2), c1 = 1 for the second-derivative reading and 2 as
printed; Eq. 5 gives d = mu -/+ (1 / (sqrt(2 pi) ln2)) / (w sigma), minus for
edges and plus for non-edges.

    python tests/golden/make_parabola_closed_forms.py   # rewrites the file
"""
import math
import os

HEADER = """# Closed-form values of the parabola parameters at delta = mu (u = 0).
# Source: Eq. 4 (w) and Eq. 5 (d), Sec. II.C; the non-edge variant flips the
# marked operators.  At u = 0, exp(-u^2/2) = 1 and 1 -/+ erf(0) = 1, so Eq. 4's
# second term vanishes and its first term is c1 / (pi ln2 sigma^2), with c1 = 1
# for the derived reading (second-derivative match) and c1 = 2 as printed.
# Eq. 5 then gives d = mu -/+ (1 / (sqrt(2 pi) ln2)) / (w sigma)
# (minus for edges, plus for non-edges).  Values below are that arithmetic
# in double precision.
# columns: reading  kind  mu  sigma  w  d
"""

CASES = [("derived", "edge", 1.5, 1.0), ("derived", "nonedge", 1.5, 1.0), ("printed", "edge", 1.5, 1.0),
         ("printed", "nonedge", 1.5, 1.0), ("derived", "edge", 1.5, 0.5), ("derived", "nonedge", 2.0, 2.0),
         ("printed", "edge", 0.7, 0.3)]


def rows():
    ln2 = math.log(2.0)
    out = []
    for reading, kind, mu, sigma in CASES:
        c1 = 1.0 if reading == "derived" else 2.0
        w = c1 / (math.pi * ln2 * sigma * sigma)
        g = (1.0 / (math.sqrt(2.0 * math.pi) * ln2)) / (w * sigma)
        d = mu - g if kind == "edge" else mu + g
        out.append(f"{reading} {kind} {mu} {sigma} {w!r} {d!r}")
    return out


def text():
    return HEADER + "\n".join(rows()) + "\n"


if __name__ == "__main__":
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "parabola_closed_forms.txt"), "w") as f:
        f.write(text())
