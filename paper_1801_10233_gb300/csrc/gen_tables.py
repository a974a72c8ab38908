"""Write sl_tables.h: the constants of the double-float exponential.

exp(x) = 2^m * 2^(j/64) * exp(r) with x = (64 m + j) ln2/64 + r, |r| <= ln2/128
(a table-driven reduction in the manner of Tang, ACM TOMS 15 (1989)).  This
script computes 2^(j/64) and ln2/64 to 50 decimal digits with Python's
decimal module and splits each into float pieces: T[j] = hi + lo (48 bits),
ln2/64 = c1 + c2 + c3 with c1 holding 14 significant bits so that n * c1 is
exact for |n| < 1024.  Run: python gen_tables.py > sl_tables.h
"""
from decimal import Decimal, getcontext

import numpy as np

getcontext().prec = 60


def f32(x):
    return np.float32(float(x))


def split2(x):
    hi = f32(x)
    lo = f32(x - Decimal(float(hi)))
    return hi, lo


def ln2():
    return Decimal(2).ln()


def hexf(v):
    return float(v).hex() + "f" if float(v) != 0.0 else "0.0f"


def main():
    out = ["// Generated by gen_tables.py: constants of the double-float exp.", "#pragma once", ""]
    out.append("// 2^(j/64) = hi + lo, j = 0..63 (global memory: lanes index it independently)")
    out.append("__device__ const float2 kSlExp2Table[64] = {")
    for j in range(64):
        x = Decimal(2) ** (Decimal(j) / Decimal(64))
        hi, lo = split2(x)
        out.append(f"  {{{hexf(hi)}, {hexf(lo)}}},")
    out.append("};")
    c = ln2() / Decimal(64)
    # c1: c rounded to 14 significant bits
    e = int(np.floor(np.log2(float(c))))
    scale = Decimal(2) ** (13 - e)
    c1 = (c * scale).to_integral_value() / scale
    rest = c - c1
    c2 = f32(rest)
    c3 = f32(rest - Decimal(float(c2)))
    inv = Decimal(64) / ln2()
    out.append("")
    out.append(f"#define SL_LN2_64_C1 {hexf(f32(c1))}  // ln2/64, first 14 bits")
    out.append(f"#define SL_LN2_64_C2 {hexf(c2)}")
    out.append(f"#define SL_LN2_64_C3 {hexf(c3)}")
    out.append(f"#define SL_64_LN2 {hexf(f32(inv))}")
    out.append("")
    out.append("// 1/k! as hi + lo, for the rotation series")
    for k in (3, 4, 5, 6):
        fac = 1
        for q in range(2, k + 1):
            fac *= q
        hi, lo = split2(Decimal(1) / Decimal(fac))
        out.append(f"#define SL_INV_FACT{k}_HI {hexf(hi)}")
        out.append(f"#define SL_INV_FACT{k}_LO {hexf(lo)}")
    out.append("")
    out.append("// ln2, 2 pi, 1/(2k+1) and 1/k! as hi + lo, for the double-float log, sincos")
    out.append("// and the Box-Muller normals of the spin bath")
    hi, lo = split2(ln2())
    out.append(f"#define SL_LN2_HI {hexf(hi)}")
    out.append(f"#define SL_LN2_LO {hexf(lo)}")
    pi = Decimal("3.14159265358979323846264338327950288419716939937510582097494459")
    hi, lo = split2(2 * pi)
    out.append(f"#define SL_2PI_HI {hexf(hi)}")
    out.append(f"#define SL_2PI_LO {hexf(lo)}")
    hi, lo = split2(Decimal(2).sqrt())
    out.append(f"#define SL_SQRT2_HI {hexf(hi)}")
    for k in range(1, 13):
        hi, lo = split2(Decimal(1) / Decimal(2 * k + 1))
        out.append(f"#define SL_INV_ODD{2 * k + 1}_HI {hexf(hi)}")
        out.append(f"#define SL_INV_ODD{2 * k + 1}_LO {hexf(lo)}")
    fac = 1
    for k in range(1, 19):
        fac *= k
        hi, lo = split2(Decimal(1) / Decimal(fac))
        out.append(f"#define SL_INV_FAC{k}_HI {hexf(hi)}")
        out.append(f"#define SL_INV_FAC{k}_LO {hexf(lo)}")
    assert float(f32(c1)) == float(c1)
    print("\n".join(out))


if __name__ == "__main__":
    main()
