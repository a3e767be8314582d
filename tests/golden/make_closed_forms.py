"""Write atm_closed_forms.txt: exact energies of two triangle shapes.

Eq. atm at side lengths (r_ij, r_ik, r_jk):
  equilateral (r, r, r):        u = nu (1 + 3/8) / r^9 = 11 nu / (8 r^9)
  collinear, equally spaced (i--j = r, i--k = 2r, j--k = r):
      1/(r^3 (2r)^3 r^3) = 1/(8 r^9),  3 (4r^2)(-2r^2)(4r^2) / (8 r^5 (2r)^5 r^5) = -3/(8 r^9)
      u = -nu / (4 r^9)
The values are computed in exact rational arithmetic and rounded once to FP64.
This script uses neither the oracle nor the CUDA library.
"""
import os
from fractions import Fraction

NUS = [Fraction(73, 1000), Fraction(72, 1000)]
RS = [Fraction(9, 10), Fraction(1), Fraction(11, 10), Fraction(5, 4), Fraction(3, 2), Fraction(2),
      Fraction(12, 5)]

out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "atm_closed_forms.txt")
with open(out, "w") as fh:
    fh.write("# Eq. atm closed forms: nu r E_equilateral(11nu/8r^9) E_collinear(-nu/4r^9)\n")
    fh.write("# exact rationals rounded to FP64 (make_closed_forms.py)\n")
    for nu in NUS:
        for r in RS:
            e_eq = nu * 11 / (8 * r ** 9)
            e_col = -nu / (4 * r ** 9)
            fh.write("%r %r %r %r\n" % (float(nu), float(r), float(e_eq), float(e_col)))
