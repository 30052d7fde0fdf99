"""Writes pbe_log_table.h, the tables of the table-driven logarithm and
exponential in pbe_math.cuh (every entry computed with 50 decimal digits,
then rounded once to the nearest double):

  log: for j = 0..255 the interval [1 + j/256, 1 + (j+1)/256) of the mantissa
       has the centre c_j = 1 + (j + 1/2)/256; PBE_LOG_TAB_INV holds 1/c_j,
       PBE_LOG_TAB_LN holds ln(c_j);
  exp: PBE_EXP_TAB holds 2^(j/64), j = 0..63; PBE_EXP_LN2_64_HI/LO split
       ln(2)/64 into a double and the double nearest to the remainder."""
import decimal
import os

decimal.getcontext().prec = 50
HERE = os.path.dirname(os.path.abspath(__file__))


def table(f, name, vals, per_line=4):
    f.write(f"#define {name} \\\n    {{ \\\n")
    for k in range(0, len(vals), per_line):
        tail = ", \\\n" if k + per_line < len(vals) else " \\\n"
        f.write("        " + ", ".join(repr(v) for v in vals[k:k + per_line]) + tail)
    f.write("    }\n")


def main():
    D = decimal.Decimal
    inv, ln = [], []
    for j in range(256):
        num = 513 + 2 * j                    # c_j = num / 512, exact
        inv.append(512.0 / num)              # one correctly rounded division
        ln.append(float((D(num) / D(512)).ln()))
    ln2 = D(2).ln()
    two_j = [float((ln2 * D(j) / D(64)).exp()) for j in range(64)]
    ln2_64 = ln2 / D(64)
    hi = float(ln2_64)
    lo = float(ln2_64 - D(hi))
    with open(os.path.join(HERE, "pbe_log_table.h"), "w") as f:
        f.write("// Generated by gen_log_table.py (50-digit arithmetic, each entry rounded once).\n")
        f.write("// PBE_LOG_TAB_INV / PBE_LOG_TAB_LN: 1/c_j and ln(c_j), c_j = 1 + (j + 1/2)/256, j = 0..255;\n")
        f.write("// PBE_EXP_TAB: 2^(j/64), j = 0..63; PBE_EXP_LN2_64_HI + PBE_EXP_LN2_64_LO = ln(2)/64.\n")
        f.write("#pragma once\n")
        table(f, "PBE_LOG_TAB_INV", inv)
        table(f, "PBE_LOG_TAB_LN", ln)
        table(f, "PBE_EXP_TAB", two_j)
        f.write(f"#define PBE_EXP_LN2_64_HI {hi!r}\n")
        f.write(f"#define PBE_EXP_LN2_64_LO {lo!r}\n")


if __name__ == "__main__":
    main()
