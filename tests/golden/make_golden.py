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

    # 1-to-1 pairs (Table II): document j as the query, document j + 1 as the target
    docs = [(C.word_ids[C.doc_ptr[j]:C.doc_ptr[j + 1]], C.vals[C.doc_ptr[j]:C.doc_ptr[j + 1]])
            for j in range(51)]
    pairs = oracle.wmd_pairs(E, docs[:50], docs[1:51], 2.0, 10)
    header = ("1-to-1 Sinkhorn WMD, FP64 oracle (cost over the target's words): workload 'tiny', "
              "pair j = (document j, document j+1), j < 50, lambda=2, t=10, seed 210706433")
    np.savetxt(os.path.join(HERE, "tiny_pairs.txt"), pairs, fmt="%.17g", header=header)


if __name__ == "__main__":
    main()
