"""Seeded synthetic inputs: codes (H in CSR form), codewords and channel LLRs.

Shared by the oracle tests and the CUDA path; contains none of the decoder's
arithmetic.  Importing this subpackage never loads the CUDA library.
"""
from .codes import (Code, from_rows, hamming74, regular_code, qc_code, staircase_code,
                    tree_code, permuted)
from .encode import Encoder, rref_gf2, syndrome
from .channel import awgn_llr, quantize, noiseless, sigma2
from .workloads import MULTI8, WORKLOADS, Workload, make_multi_workload, make_workload, multi8_frame_counts

__all__ = ["Code", "from_rows", "hamming74", "regular_code", "qc_code", "staircase_code",
           "tree_code", "permuted", "Encoder", "rref_gf2", "syndrome", "awgn_llr",
           "quantize", "noiseless", "sigma2", "WORKLOADS", "make_workload", "Workload", "MULTI8",
           "make_multi_workload", "multi8_frame_counts"]
