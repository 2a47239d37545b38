"""Writes the oracle-derived golden fixtures in this directory.

Calls only ``oracle/`` (and the seeded input generators).  Run from the
repository root:  python tests/golden/make_golden.py
"""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O                      # noqa: E402
from paper_1905_06850_gb300 import workloads as W   # noqa: E402


def main():
    c = W.config_2d()
    with open(os.path.join(HERE, "config2d_iters.txt"), "w") as f:
        f.write("# 2D 5-point Laplacian 100x100, x* ~ U[-1,1] (numpy default_rng(1)), b = A x*,\n")
        f.write("# x0 = 0, Chebyshev shifts on [0, 8], 2l+1 dots; k of the returned iterate.\n")
        f.write("# Written by tests/golden/make_golden.py from the FP64 oracle.\n")
        for rtol in (1e-6, 1e-8):
            f.write(f"cg {rtol:.0e} {O.cg(c['op'], c['b'], rtol=rtol).iters}\n")
            for l in range(1, 6):
                r = O.plcg(c["op"], c["b"], l=l, sigma=O.chebyshev_shifts(l, 0, 8), rtol=rtol)
                f.write(f"plcg{l} {rtol:.0e} {r.iters}\n")
    with open(os.path.join(HERE, "spectrum_2d_100.txt"), "w") as f:
        f.write("# Extreme eigenvalues of the 100x100 Dirichlet 5-point Laplacian (4, -1):\n")
        f.write("# 4 - 4 cos(pi/101) and 4 + 4 cos(pi/101) (separable closed form of the\n")
        f.write("# Kronecker sum of two 1D (2, -1) Laplacians, eigenvalues 2 - 2 cos(j pi/(N+1))).\n")
        f.write(f"lambda_min {4 - 4 * math.cos(math.pi / 101):.17g}\n")
        f.write(f"lambda_max {4 + 4 * math.cos(math.pi / 101):.17g}\n")


if __name__ == "__main__":
    main()
