"""Write tests/golden/opcounts.json: the mean algorithmic operation counts per matrix of the
method (additions, multiplications, fmas, divisions, correctly rounded hypots, eq. (EXT)
evaluations, square roots) on samples of the benchmark workloads, counted by the oracle;
the *_ncr entries count the variant with a hypot that is not correctly rounded (Alg. 1's
branch for it).

These are the "units of work" of the roofline in bench.py: the method's own operations as
written in Sect. 3 (exact power-of-two scalings, comparisons and sign changes excluded).
Run: python tests/golden/make_opcounts.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2407_13116_gb300 import inputs as I  # noqa: E402

SEED = 0x240713116
SAMPLE = 1 << 16


def main():
    out = {"sample": SAMPLE, "seed_base": SEED, "workloads": {}}
    for prec in ("d", "s"):
        out["workloads"]["wide_%s_gesvd2" % prec] = oracle.opcount(
            I.general(SAMPLE, SEED + 2, prec, "wide"), prec)
        out["workloads"]["wide_%s_trsvd2" % prec] = oracle.opcount(
            I.triangular(SAMPLE, SEED + 3, prec, "wide"), prec, triangular=True)
        out["workloads"]["wide_%s_gesvd2_ncr" % prec] = oracle.opcount(
            I.general(SAMPLE, SEED + 2, prec, "wide"), prec, ncr=True)
        out["workloads"]["wide_%s_trsvd2_ncr" % prec] = oracle.opcount(
            I.triangular(SAMPLE, SEED + 3, prec, "wide"), prec, triangular=True, ncr=True)
        out["workloads"]["narrow_%s_gesvd2" % prec] = oracle.opcount(
            I.general(SAMPLE, SEED + 1, prec, "narrow"), prec)
        # complex matrices (Sect. 3.4): real and imaginary planes from two wide-range streams
        G8 = np.empty((8, SAMPLE), np.float64 if prec == "d" else np.float32)
        G8[0::2] = I.general(SAMPLE, SEED + 6, prec, "wide")
        G8[1::2] = I.general(SAMPLE, SEED + 7, prec, "wide")
        out["workloads"]["wide_%s_cgesvd2" % prec] = oracle.opcount(G8, prec, complex_planes=True)
    with open(os.path.join(HERE, "opcounts.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
