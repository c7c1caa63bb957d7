"""Writes ssss_closed_form.txt: textbook closed forms for [ss|ss] (no oracle, no CUDA path).

R = 0: four identical normalised s Gaussians on one centre give 2 sqrt(alpha/pi).
R > 0: A = B, C = D, equal exponents: two unit Gaussian charges of exponent 2 alpha,
whose Coulomb energy is erf(sqrt(alpha) R) / R.
"""
import math
import os

ROWS = [(1.0, 0.0), (1.0, 1.0), (1.0, 2.5), (0.5, 3.0)]


def value(alpha, R):
    return 2 * math.sqrt(alpha / math.pi) if R == 0 else math.erf(math.sqrt(alpha) * R) / R


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ssss_closed_form.txt")
    with open(path, "w") as f:
        f.write("# Closed forms for [ss|ss] of arXiv 2303.13632 Eq. 1 with normalised s functions (Sec. II-A):\n")
        f.write("# A = B = origin, C = D = (0, 0, R), one exponent alpha for all four functions.\n")
        f.write("# R = 0: 2 sqrt(alpha/pi); R > 0: two unit Gaussian charges of exponent 2 alpha interact\n")
        f.write("# as erf(sqrt(alpha) R) / R (textbook electrostatics, independent of any ERI recursion).\n")
        f.write("# Written by make_ssss_closed_form.py.\n")
        f.write("# alpha   R     value\n")
        for a, R in ROWS:
            f.write(f"{a!r} {R!r} {value(a, R)!r}\n")


if __name__ == "__main__":
    main()
