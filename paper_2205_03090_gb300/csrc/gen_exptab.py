"""Writes ptf_exptab.cuh: the table of the device exponential.

ptf::exp_fast writes x = (64 m + j) ln2/64 + r with |r| <= ln2/128 and
evaluates e^x = 2^m 2^(j/64) e^r (the table-driven method of P. T. P. Tang,
ACM TOMS 15 (1989) 144).  The table holds 2^(j/64), j = 0..63, and the
reduction constant ln2/64 split as L1 + L2, L1 with its low 20 significand
bits zero (so n L1 is exact for |n| < 2^20); all rounded to double from
200-bit values.  Run: python gen_exptab.py > ptf_exptab.cuh
"""
import mpmath

mpmath.mp.prec = 200
c = mpmath.log(2) / 64
L1 = float(c)
b = int.from_bytes(__import__("struct").pack(">d", L1), "big") & ~((1 << 20) - 1)
L1 = __import__("struct").unpack(">d", b.to_bytes(8, "big"))[0]
L2 = float(c - mpmath.mpf(L1))
inv = float(64 / mpmath.log(2))
print("// ptf_exptab.cuh -- generated by gen_exptab.py; do not edit.")
print("// 2^(j/64), j = 0..63, and ln2/64 = L1 + L2 for the table-driven exponential.")
print("#pragma once")
print("namespace ptf {")
print(f"constexpr double kExpInvL = {inv!r};   // 64 / ln 2")
print(f"constexpr double kExpL1 = {L1!r};   // ln2/64, high part")
print(f"constexpr double kExpL2 = {L2!r};   // ln2/64 - L1")
print("static __device__ const double kExpTab[64] = {")
for j in range(64):
    print(f"    {float(mpmath.power(2, mpmath.mpf(j) / 64))!r},")
print("};")
print("}  // namespace ptf")
