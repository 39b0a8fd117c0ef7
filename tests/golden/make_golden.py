"""Writes the stored oracle outputs under tests/golden/.

Calls only the oracle and the seeded input generator; no value here comes from
the CUDA path.  Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2107_06433_gb300 import synth  # noqa: E402


def main():
    E, C, (qi, qw) = synth.make("tiny")
    rp, col, val = C.csr()
    wmd = oracle.wmd(E, rp, col, val, C.N, qi, qw, 1.0, 15, "sparse")
    header = ("Sinkhorn WMD, FP64 oracle (Algorithm 1, sparse mode): workload 'tiny' "
              "(V=2000, d=64, N=200, v_r=8, lambda=1, t=15), seed 210706433")
    np.savetxt(os.path.join(HERE, "tiny_wmd.txt"), wmd, fmt="%.17g", header=header)


if __name__ == "__main__":
    main()
