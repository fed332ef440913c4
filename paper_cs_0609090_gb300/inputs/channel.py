"""BPSK over AWGN and LLR quantization (inputs only; no decoder arithmetic).

Section II of the paper: y_n = (-1)^{x_n} + xi_n and the channel LLR
Z0_n = 2 y_n / sigma^2.  For a code of rate R at Eb/N0 (dB),
sigma^2 = 1 / (2 R 10^{EbN0/10}).  Fixed-point decoders take
q_n = clamp(round_half_away(Z0_n / delta), -Qc, Qc) in int8.
"""
from __future__ import annotations

import numpy as np


def sigma2(ebn0_db: float, rate: float) -> float:
    return 1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))


def awgn_llr(codewords: np.ndarray, ebn0_db, rate: float, seed: int) -> np.ndarray:
    """Channel LLRs (float64 [F, N]) for BPSK codewords.  ``ebn0_db`` is a scalar
    or one value per frame."""
    cw = np.asarray(codewords, dtype=np.uint8)
    F, N = cw.shape
    e = np.broadcast_to(np.asarray(ebn0_db, dtype=np.float64).reshape(-1, 1), (F, 1))
    s2 = 1.0 / (2.0 * rate * 10.0 ** (e / 10.0))
    rng = np.random.Generator(np.random.Philox(key=seed))
    y = (1.0 - 2.0 * cw) + np.sqrt(s2) * rng.standard_normal((F, N))
    return 2.0 * y / s2


def quantize(llr: np.ndarray, delta: float, qc: int) -> np.ndarray:
    """int8 LLRs: round half away from zero of llr/delta, saturated to +-qc."""
    x = np.asarray(llr, dtype=np.float64) / delta
    r = np.sign(x) * np.floor(np.abs(x) + 0.5)
    return np.clip(r, -qc, qc).astype(np.int8)


def noiseless(codewords: np.ndarray, qc: int) -> np.ndarray:
    """Noise-free quantized frames: +qc for bit 0, -qc for bit 1."""
    return np.where(np.asarray(codewords) == 0, qc, -qc).astype(np.int8)
