"""Writes exp_table.h: the constants of the table-driven exponential (Tang, ACM TOMS 15(2), 1989).

exp(x) = 2^(n / 64) exp(r) with n = round(64 x / ln 2) and r = x - n ln 2 / 64; 2^(n / 64) splits
into 2^(n div 64), applied to the exponent field, and a 64-entry table of 2^(j / 64), j = 0..63.
Every constant is computed here in 60-digit decimal arithmetic and rounded once to the nearest
double (Python's float() of a Decimal is correctly rounded), so the header is reproducible
bit for bit on any host.  Run:  python gen_exp_table.py > exp_table.h
"""
from decimal import Decimal, getcontext

getcontext().prec = 60


def hexd(v: Decimal) -> str:
    return float(v).hex()


def main() -> None:
    ln2 = Decimal(2).ln()
    step = ln2 / 64
    hi = Decimal(float(step))
    lo = step - hi
    out = ["// Generated by gen_exp_table.py; do not edit.",
           "// Constants of the table-driven exponential (Tang, ACM TOMS 15(2), 1989):",
           "// 64 / ln 2, ln 2 / 64 as a double-double, and 2^(j / 64) for j = 0..63, each the",
           "// double nearest to the exact value.",
           "#pragma once",
           "namespace chem {",
           f"constexpr double kExpInvStep = {hexd(64 / ln2)};   // 64 / ln 2",
           f"constexpr double kExpStepHi = {hexd(hi)};   // ln 2 / 64, leading part",
           f"constexpr double kExpStepLo = {hexd(lo)};   // ln 2 / 64 - kExpStepHi",
           "#define CHEM_EXP_TABLE_VALUES \\"]
    vals = [hexd((Decimal(j) / 64 * ln2).exp()) for j in range(64)]
    for i in range(0, 64, 4):
        out.append("    " + ", ".join(vals[i:i + 4]) + ("," if i + 4 < 64 else "") + " \\")
    out.append("")
    out.append("constexpr double kExpTable[64] = {CHEM_EXP_TABLE_VALUES};")
    out.append("}  // namespace chem")
    print("\n".join(out))


if __name__ == "__main__":
    main()
