"""Writes the regression fixtures of tests/golden from the CPU oracle only.

Run from the repository root:  python tests/golden/make_golden.py
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import bsrht  # noqa: E402


def main():
    om = bsrht.dense_omega(16, 4, 8, 0)
    path = os.path.join(HERE, "omega_n16_p4_l8_seed0.txt")
    header = ("Signs of the block SRHT Omega (n=16, p=4, l=8, seed=0); every entry "
              "is sign/sqrt(8). Written by make_golden.py from the oracle.")
    np.savetxt(path, np.sign(om).astype(np.int64), fmt="%d", header=header)


if __name__ == "__main__":
    main()
