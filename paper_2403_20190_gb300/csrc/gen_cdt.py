"""Writes cdt_table.h: thresholds of the discrete Gaussian used for RLWE/RGSW
errors (sigma = 3.2, support |x| <= 19, probabilities proportional to
exp(-x^2 / (2 sigma^2))).  Threshold i is floor(2^63 * P(X <= -19 + i)) for
i = 0..37, computed with the standard library's decimal arithmetic at 60
significant digits.  Run: python gen_cdt.py > cdt_table.h
"""
from decimal import Decimal, getcontext

getcontext().prec = 60
SIGMA = Decimal("3.2")
SUPPORT = 19


def thresholds():
    two_s2 = 2 * SIGMA * SIGMA
    rho = [(-(Decimal(x) * Decimal(x)) / two_s2).exp() for x in range(-SUPPORT, SUPPORT + 1)]
    z = sum(rho, Decimal(0))
    scale = Decimal(2) ** 63
    out, run = [], Decimal(0)
    for i in range(2 * SUPPORT):
        run += rho[i]
        out.append(int((scale * run / z).to_integral_value(rounding="ROUND_FLOOR")))
    return out


def main():
    t = thresholds()
    print("// Generated by gen_cdt.py -- discrete Gaussian (sigma = 3.2) inversion table.")
    print("#pragma once")
    print("#include <cstdint>")
    print(f"#define HW_CDT_LEN {len(t)}")
    print(f"#define HW_CDT_SUPPORT {SUPPORT}")
    print("#define HW_CDT_VALUES \\")
    rows = [", ".join(f"{v}ULL" for v in t[i:i + 3]) for i in range(0, len(t), 3)]
    for k, row in enumerate(rows):
        print("    " + row + (", \\" if k + 1 < len(rows) else ""))


if __name__ == "__main__":
    main()
