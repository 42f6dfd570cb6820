"""Writes lotkin_cond1.txt: log10 of ||A||_1, ||A^-1||_1 and their product
for the n x n Lotkin matrix of Sec. 4 (first row ones, a_ij = 1/(i+j-1)
below), computed exactly by the oracle (oracle.lotkin_norm1_log2: the
integer inverse of the Hilbert matrix and the Sherman-Morrison update, in
Python integers).  Sec. 4 prints 4.3e1576 for ||A||_1 ||A^-1||_1 at
n = 1024; the exact value is 3.129e1565.

    python tests/golden/make_lotkin_cond1.py
"""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as orc  # noqa: E402


def main():
    lines = ["# n log10_norm1_A log10_norm1_inverse log10_cond1 (exact; written by make_lotkin_cond1.py)"]
    for n in (64, 256, 1024):
        la, li = orc.lotkin_norm1_log2(n)
        k = math.log10(2.0)
        lines.append("%d %.6f %.6f %.6f" % (n, la * k, li * k, (la + li) * k))
    with open(os.path.join(HERE, "lotkin_cond1.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
