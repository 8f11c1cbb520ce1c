"""Writes ftrans_figS1.txt: f_trans (Eq. S1) evaluated in exact rational
arithmetic at the two parameter sets plotted in Fig. S1, f(x, 2, 4) and
f(x, 1, 6).  The coefficients 0.9375, 0.625, 0.1875 are the ones printed in
Eq. S1 (15/16, 5/8, 3/16); no other code is used."""
from fractions import Fraction as Q
import os


def f(x, lo, hi):
    if x <= lo:
        return Q(1)
    if x >= hi:
        return Q(0)
    t = (hi + lo - 2 * x) / (hi - lo)
    return Q(1, 2) + Q(15, 16) * t - Q(5, 8) * t**3 + Q(3, 16) * t**5


rows = []
for lo, hi in ((2, 4), (1, 6)):
    for k in range(0, 57):
        x = Q(k, 8)
        rows.append((lo, hi, x, f(x, Q(lo), Q(hi))))
here = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(here, "ftrans_figS1.txt"), "w") as fh:
    fh.write("# f_trans(x, lo, hi), Eq. S1, at the Fig. S1 parameter sets; exact rationals\n")
    fh.write("# lo hi x_num/x_den f_num/f_den\n")
    for lo, hi, x, v in rows:
        fh.write(f"{lo} {hi} {x.numerator}/{x.denominator} {v.numerator}/{v.denominator}\n")
