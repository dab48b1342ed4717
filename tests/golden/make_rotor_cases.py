"""Writes rotor_cases.txt: rotors whose rotation matrix has a closed form.

A rotor cos(a) + sin(a) e_ij rotates the (i, j) plane by 2a (e_i -> cos 2a e_i
- sin 2a e_j) under u -> r u r^dagger (appendix A.2); the product of two such
rotors in orthogonal planes commutes and rotates both planes, its e0123 part
being the product of the two sines (e01 e23 = e0123, e02 e13 = -e0123,
e03 e12 = e0123). Nothing here calls the renderer or the oracle: the matrices
are the closed forms. Row format: 8 rotor components in storage order
(s, b01, b02, b12, b03, b13, b23, p), then the 16 matrix entries row-major.
"""
import math
import os

import numpy as np

SLOT = {(0, 1): 1, (0, 2): 2, (1, 2): 3, (0, 3): 4, (1, 3): 5, (2, 3): 6}


def givens(i, j, a):
    E = np.eye(4)
    c, s = math.cos(2 * a), math.sin(2 * a)
    E[i, i] = E[j, j] = c
    E[i, j] = s
    E[j, i] = -s
    return E


def single(i, j, a, scale=1.0):
    r = np.zeros(8)
    r[0] = math.cos(a)
    r[SLOT[(i, j)]] = math.sin(a)
    return r * scale, givens(i, j, a)


def double(p1, a, p2, b, sign):
    r = np.zeros(8)
    r[0] = math.cos(a) * math.cos(b)
    r[SLOT[p1]] = math.sin(a) * math.cos(b)
    r[SLOT[p2]] = math.cos(a) * math.sin(b)
    r[7] = sign * math.sin(a) * math.sin(b)
    return r, givens(*p1, a) @ givens(*p2, b)


def main():
    cases = [
        (np.array([1.0, 0, 0, 0, 0, 0, 0, 0]), np.eye(4)),
        single(0, 1, math.pi / 8),
        single(0, 3, math.pi / 6),
        single(2, 3, -0.4),
        single(1, 2, 0.7, scale=3.0),
        double((0, 1), 0.3, (2, 3), 0.5, +1.0),
        double((0, 2), -0.2, (1, 3), 0.6, -1.0),
        double((0, 3), 0.45, (1, 2), -0.35, +1.0),
    ]
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rotor_cases.txt")
    with open(path, "w") as f:
        f.write("# rotor (s b01 b02 b12 b03 b13 b23 p) then R row-major; closed forms, "
                "appendix A.2 (u' = r u r^dagger). Written by make_rotor_cases.py\n")
        for r, R in cases:
            f.write(" ".join(f"{x:.17g}" for x in list(r) + list(R.flatten())) + "\n")


if __name__ == "__main__":
    main()
