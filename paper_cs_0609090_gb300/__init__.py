"""GB300 (sm_103a) single-scan min-sum LDPC decoder.

Subpackages:
  inputs  - seeded codes, codewords and channel LLRs (no CUDA needed)
  ldpc    - thin ctypes binding over the C-ABI library libldpc_gb300.so
            (import it explicitly; it fails loudly if the library is missing)
"""
__version__ = "0.1.0"
