"""Writes brick_unit_cube.txt: closed-form Nedelec brick matrices (unit cube).

Hand derivation with exact fractions, independent of the quadrature used by
the oracle.  Edge functions: x-edge (a, b) = x^ phi_a(y) phi_b(z), y-edge
(a, b) = y^ phi_a(x) phi_b(z), z-edge (a, b) = z^ phi_a(x) phi_b(y), with
phi_0 = 1 - t, phi_1 = t and local order (a, b) = (0,0), (1,0), (0,1), (1,1).
1-D integrals: int phi_a phi_b = m_ab (1/3 diagonal, 1/6 off), phi_a' = s_a
(s_0 = -1, s_1 = +1).  Curls: x(a,b) -> (0, phi_a(y) s_b, -s_a phi_b(z));
y(a,b) -> (-phi_a(x) s_b, 0, s_a phi_b(z)); z(a,b) -> (phi_a(x) s_b,
-s_a phi_b(y), 0).
"""
import os
from fractions import Fraction as Fr

m = {(0, 0): Fr(1, 3), (1, 1): Fr(1, 3), (0, 1): Fr(1, 6), (1, 0): Fr(1, 6)}
s = {0: -1, 1: 1}
off = [(0, 0), (1, 0), (0, 1), (1, 1)]


def matrices():
    M = [[Fr(0)] * 12 for _ in range(12)]
    S = [[Fr(0)] * 12 for _ in range(12)]
    for f in range(3):
        for i, (a, b) in enumerate(off):
            for j, (a2, b2) in enumerate(off):
                M[4 * f + i][4 * f + j] = m[a, a2] * m[b, b2]
                S[4 * f + i][4 * f + j] = m[a, a2] * s[b] * s[b2] + s[a] * s[a2] * m[b, b2]
    for i, (a, b) in enumerate(off):
        for j, (a2, b2) in enumerate(off):
            xy = -s[a] * s[a2] * m[b, b2]      # z-components: -s_a phi_b(z) * s_a2 phi_b2(z)
            xz = -s[b] * s[a2] * m[a, b2]      # y-components: phi_a(y) s_b * (-s_a2 phi_b2(y))
            yz = -s[b] * s[b2] * m[a, a2]      # x-components: -phi_a(x) s_b * phi_a2(x) s_b2
            S[i][4 + j] = S[4 + j][i] = xy
            S[i][8 + j] = S[8 + j][i] = xz
            S[4 + i][8 + j] = S[8 + j][4 + i] = yz
    return M, S


if __name__ == "__main__":
    M, S = matrices()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "brick_unit_cube.txt")
    with open(path, "w") as fh:
        fh.write("# Closed-form lowest-order Nedelec brick matrices on the unit cube, x 36.\n")
        fh.write("# Written by make_brick_unit_cube.py (hand derivation, exact fractions).\n")
        for name, X in (("M", M), ("S", S)):
            fh.write(name + "\n")
            for r in X:
                fh.write(" ".join(str(int(v * 36)) for v in r) + "\n")
