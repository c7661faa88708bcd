"""Write drt_fnodes.h: the UTD transition function F(X) at the nodes X_i = 6 + i / 2, i = 0..68.

F(X) = 2j sqrt(X) exp(jX) int_{sqrt X}^inf exp(-j t^2) dt = sqrt(pi X) exp(j pi/4) erfcx(z),
z = exp(j pi/4) sqrt(X), with erfcx from its Laplace continued fraction
erfcx(z) = 1 / (sqrt(pi) (z + (1/2) / (z + 1 / (z + (3/2) / (z + ...))))) evaluated bottom-up in
50-digit decimal arithmetic to depth 3000 (the result does not change at depth 6000).  The device
code expands F around the nearest node by its Taylor series (F' = F (1/(2X) + j) - j).

  python paper_2205_00237_gb300/csrc/gen_fnodes.py     # rewrites drt_fnodes.h beside this script
"""
import os
from decimal import Decimal as D, getcontext

getcontext().prec = 50
X0, H, NN = 6, 2, 69   # X_i = X0 + i / H
SQPI = D("1.7724538509055160272981674833411451827975494561223871282138")


def F(X, depth=3000):
    X = D(X)
    r2 = D(2).sqrt() / 2
    sx = X.sqrt()
    zr = zi = r2 * sx
    fr, fi = zr, zi
    for k in range(depth, 0, -1):
        a = D(k) / 2
        den = fr * fr + fi * fi
        fr, fi = zr + a * fr / den, zi - a * fi / den
    pr = pi_ = SQPI * sx * r2
    br, bi = fr * SQPI, fi * SQPI
    den = br * br + bi * bi
    return (pr * br + pi_ * bi) / den, (pi_ * br - pr * bi) / den


def main():
    rows = []
    for i in range(NN):
        re, im = F(D(X0) + D(i) / H)
        rows.append(f"    {float(re).hex()}, {float(im).hex()},   // X = {X0 + i / H}")
    src = (
        "// Generated by gen_fnodes.py: the UTD transition function F(X) (re, im) at X_i = 6 + i / 2,\n"
        "// i = 0..68, from its continued fraction in 50-digit arithmetic.\n#pragma once\n\n"
        "namespace drt {\n\nconstexpr double FNODE_X0 = 6.0, FNODE_H = 0.5;\nconstexpr int FNODE_N = 69;\n"
        "static __device__ const double kFnode[2 * FNODE_N] = {\n" + "\n".join(rows) + "\n};\n\n}  // namespace drt\n")
    open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "drt_fnodes.h"), "w").write(src)


if __name__ == "__main__":
    main()
