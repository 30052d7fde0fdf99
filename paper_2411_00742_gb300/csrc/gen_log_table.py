"""Writes pbe_log_table.h, the table of the table-driven logarithm in
pbe_math.cuh: for j = 0..127 the interval [1 + j/128, 1 + (j+1)/128) of the
mantissa has the centre c_j = 1 + (j + 1/2)/128; the table holds the double
nearest to 1/c_j and the double nearest to ln(c_j) (computed with 50 decimal
digits, then rounded once)."""
import decimal
import os

decimal.getcontext().prec = 50
HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    inv, ln = [], []
    for j in range(128):
        num = 257 + 2 * j                    # c_j = num / 256, exact
        inv.append(256.0 / num)              # one correctly rounded division
        ln.append(float((decimal.Decimal(num) / decimal.Decimal(256)).ln()))
    with open(os.path.join(HERE, "pbe_log_table.h"), "w") as f:
        f.write("// Generated by gen_log_table.py: c_j = 1 + (j + 1/2)/128, j = 0..127;\n")
        f.write("// PBE_LOG_TAB_INV: nearest double to 1/c_j; PBE_LOG_TAB_LN: nearest double to ln(c_j).\n")
        f.write("#pragma once\n")
        for name, vals in (("PBE_LOG_TAB_INV", inv), ("PBE_LOG_TAB_LN", ln)):
            f.write(f"#define {name} \\\n    {{ \\\n")
            for k in range(0, 128, 4):
                f.write("        " + ", ".join(repr(v) for v in vals[k:k + 4]) + (", \\\n" if k + 4 < 128 else " \\\n"))
            f.write("    }\n")


if __name__ == "__main__":
    main()
