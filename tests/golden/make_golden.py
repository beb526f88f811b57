"""Writes the stored expected values under tests/golden/ by calling only the
oracle (no GPU, no library).

m5inv_b1.5_c0.5_M51.8_m0.002_Ls12.txt: M5op^-1 per chirality (Sec. 2.2: the
fifth-dimension block M5op = A + B P of the even-odd form, with the Mobius
reading of M5 and the wrap terms times -mass), at the fifth-dimension
parameters of the 16^3x32 workload; rows s, columns t, chirality 0 (spins
0, 1) then chirality 1 (spins 2, 3), 17 significant digits.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

PARAMS = dict(b=1.5, c=0.5, M5=1.8, mass=0.002, Ls=12)
NAME = "m5inv_b1.5_c0.5_M51.8_m0.002_Ls12.txt"


def compute():
    p = PARAMS
    U = np.zeros((16, 4, 3, 3), dtype=np.complex128)
    for mu in range(4):
        U[:, mu] = np.eye(3)
    o = oracle.Oracle((2, 2, 2, 2), p["Ls"], p["b"], p["c"], p["M5"], p["mass"], U)
    return [o.m5inv_closed(chi) for chi in (0, 1)]


def main():
    mats = compute()
    with open(os.path.join(HERE, NAME), "w") as f:
        f.write("# M5op^-1 (Sec. 2.2), b=1.5 c=0.5 M5=1.8 mass=0.002 Ls=12; written by make_golden.py (oracle only)\n")
        for chi, M in enumerate(mats):
            f.write(f"# chirality {chi}\n")
            for row in M:
                f.write(" ".join(f"{v:.17g}" for v in row) + "\n")


if __name__ == "__main__":
    main()
