"""Oracle for the enhanced Kogbetliantz SVD of order two (arXiv 2407.13116).

TEST INFRASTRUCTURE ONLY.  A plain, slow CPU implementation written from the
paper (plain C, explicit fma, binary128 for the wide type of eq. (EXT)), with a
numpy front end.  It shares no code with the CUDA path.  Only tests/, the smoke
check and the CPU-baseline leg of bench.py may import it.

Functions whose result is not pinned by an independent check are marked
"parity unpinned" in their docstrings.
"""
from .k2ref import (build, lib, gesvd2, trsvd2, cgesvd2, hypot, hypot_n, hypot_ncr, hypot_ncr_n, prescale2, lasv2, trace, efops, prec, effl, ext,
                    brute_sigma, dmetrics, FLAGS, opcount, OPS, gesvd2_bwd, kogbet, kog_sigma_bwd, gesvdr, dyn_pairs)

__all__ = ["build", "lib", "gesvd2", "trsvd2", "cgesvd2", "hypot", "hypot_n", "hypot_ncr", "hypot_ncr_n", "prescale2", "lasv2", "trace", "efops", "prec", "effl",
           "ext", "brute_sigma", "dmetrics", "FLAGS", "opcount", "OPS", "gesvd2_bwd", "kogbet", "kog_sigma_bwd", "gesvdr", "dyn_pairs"]
