"""Writes ptf_logtab.cuh: the breakpoint table of the device logarithm.

ptf::log_fast reduces x = 2^e m with m in [0.75, 1.5), picks the nearest
breakpoint F_j = 0.75 + j/128 (j = 0..96) and evaluates
ln x = e ln 2 + ln F_j + ln(1 + r), r = (m - F_j) / F_j, |r| <= 1/192
(the table-driven reduction of P. T. P. Tang, ACM TOMS 16 (1990) 378).
For each j the table holds 1/F_j and ln F_j, rounded to double by the host
libm.  Run: python gen_logtab.py > ptf_logtab.cuh
"""
import math

rows = []
for j in range(97):
    F = 0.75 + j / 128.0
    rows.append((1.0 / F, math.log(F)))
print("// ptf_logtab.cuh -- generated by gen_logtab.py; do not edit.")
print("// Breakpoints F_j = 0.75 + j/128, j = 0..96: {1/F_j, ln F_j}.")
print("#pragma once")
print("namespace ptf {")
print("static __device__ const double kLogTab[97][2] = {")
for a, b in rows:
    print(f"    {{{a!r}, {b!r}}},")
print("};")
print("}  // namespace ptf")
