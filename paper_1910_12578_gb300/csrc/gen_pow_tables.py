"""Write sdc_pow_tables.h: the tables and polynomial coefficients of the
table-driven base-2 logarithm and exponential that the Newton kernels use for
the power-law rate factors T^nu = 2^(nu log2 T).

Method: P. T. P. Tang's table-driven reductions (ACM TOMS 15 (1989) 144-157
for the exponential, 16 (1990) 378-400 for the logarithm):
  log2 x = e + log2(1/c_j) + log2(1 + r),  x = 2^e m, m in [1, 2),
           j = the top 7 fraction bits of m, c_j = 1/(1 + (j + 1/2)/128),
           r = m c_j - 1 (one FMA, |r| <= 1/255);
  2^y    = 2^k 2^(i/256) 2^r,  256 y = 256 k + i + 256 r,  |r| <= 1/512.
The polynomials are the Taylor series, truncated where the remainder drops
below 4e-17: log2(1 + r) = sum_{n=1..6} (-1)^(n+1) r^n / (n ln 2) and
2^r - 1 = sum_{n=1..4} (r ln 2)^n / n!.  Every constant is computed here in
60-digit decimal arithmetic and rounded once to double; log2(1/c_j) is split
into a double and the double nearest its remainder.

Run from this directory:  python gen_pow_tables.py > sdc_pow_tables.h
"""
from decimal import Decimal, getcontext

getcontext().prec = 60


def d2h(x):
    """Decimal -> nearest double, as a C hex literal."""
    return float(x).hex()


def ln(x):
    return Decimal(x).ln()


LN2 = ln(2)


def log2(x):
    return ln(x) / LN2


def exp2(x):
    return (Decimal(x) * LN2).exp()


def main():
    out = []
    out.append("// sdc_pow_tables.h -- generated by gen_pow_tables.py (do not edit): tables and Taylor")
    out.append("// coefficients of the table-driven log2 / exp2 (Tang's reductions) behind T^nu = 2^(nu log2 T).")
    out.append("#pragma once")
    out.append("")
    out.append("namespace sdcd {")
    out.append("")
    out.append("// 2^(i/256), i = 0..255")
    out.append("__device__ const double POW_EXP2_T[256] = {")
    out.append(",\n".join("    " + d2h(exp2(Decimal(i) / 256)) for i in range(256)))
    out.append("};")
    cs, his, los = [], [], []
    for j in range(128):
        c = float(1 / (1 + (Decimal(j) + Decimal("0.5")) / 128))   # c_j, rounded to double
        v = log2(1 / Decimal(c))                                     # log2(1/c_j) of that double
        hi = float(v)
        lo = float(v - Decimal(hi))
        cs.append(c.hex())
        his.append(hi.hex())
        los.append(lo.hex())
    out.append("// c_j = 1/(1 + (j + 1/2)/128) and log2(1/c_j) = hi + lo, j = 0..127")
    for name, vals in (("POW_LOG_C", cs), ("POW_LOG_HI", his), ("POW_LOG_LO", los)):
        out.append("__device__ const double %s[128] = {" % name)
        out.append(",\n".join("    " + v for v in vals))
        out.append("};")
    out.append("// log2(1 + r) = r (a1 + r (a2 + ... + r a6)),  a_n = (-1)^(n+1) / (n ln 2)")
    for n in range(1, 7):
        out.append("constexpr double POW_LOG_A%d = %s;" % (n, d2h(Decimal((-1) ** (n + 1)) / (n * LN2))))
    out.append("// 2^r - 1 = r (b1 + r (b2 + r (b3 + r b4))),  b_n = (ln 2)^n / n!")
    f = Decimal(1)
    for n in range(1, 5):
        f *= n
        out.append("constexpr double POW_EXP_B%d = %s;" % (n, d2h(LN2 ** n / f)))
    out.append("")
    out.append("}  // namespace sdcd")
    print("\n".join(out))


if __name__ == "__main__":
    main()
