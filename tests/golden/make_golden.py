"""Write the oracle's FP64 cost tables used by the LUT and cost parity tests.

Calls only the CPU oracle (oracle/).  For each number of looks L it stores
100*c (Eq. 4, before flooring) and the floored int16 table on the 128 (coherence)
x 256 (slope) bin-centre grid, 100*ln(P0/P+) in fp32 for interpolated lookup,
built with an 8192-interval half grid in phase and
eight Gauss-Legendre panels per unit of -log(1-gamma).  At these settings the
oracle's P0 and P+ agree with an independent quadrature of Eqs. 5-7 to about
1e-7 relative or better (tests/test_oracle_lut.py), i.e. 100*c to about 1e-5.
Run:

    python tests/golden/make_golden.py            # all L
    python tests/golden/make_golden.py 9 50       # selected L
"""
from __future__ import annotations

import os
import sys
import time
from multiprocessing import get_context

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
LOOKS = [4.0, 6.0, 9.0, 16.0, 50.0]
NH = 8192
LAMBDA_PANELS = 8


def path_for(L: float) -> str:
    return os.path.join(HERE, f"lut_oracle_L{L:g}.npz")


def _one(L: float):
    sys.path.insert(0, ROOT)
    import oracle

    t = time.time()
    nh = NH
    cost100, table, ratio100 = oracle.lut_build(L, nh=nh, lambda_panels=LAMBDA_PANELS)
    np.savez_compressed(path_for(L), cost100=cost100, table=table, ratio100=ratio100, nlooks=L, nh=nh,
                        lambda_panels=LAMBDA_PANELS)
    return L, time.time() - t


def main(argv):
    looks = [float(a) for a in argv] or LOOKS
    sys.path.insert(0, ROOT)
    import oracle

    oracle.build()
    with get_context("spawn").Pool(len(looks)) as pool:
        for L, dt in pool.imap_unordered(_one, looks):
            print(f"L={L:g}: {dt:.0f} s -> {path_for(L)}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
