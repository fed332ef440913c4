"""Exhaustive decoders for tiny codes (N <= 20) -- TEST INFRASTRUCTURE ONLY.

Used to pin the min-sum oracle against results that do not depend on it:
  * the set of all codewords (every x in {0,1}^N with H x^T = 0, Section II);
  * the maximum-likelihood codeword for BPSK/AWGN channel values q0
    (maximises the correlation sum_n (1 - 2 x_n) q0_n);
  * the max-marginals  1/2 [max_{x: x_n = 0} corr(x) - max_{x: x_n = 1} corr(x)],
    which min-sum reaches exactly on cycle-free Tanner graphs (Wiberg's thesis).
"""
from __future__ import annotations

import numpy as np


def codewords(n_vars: int, rows) -> np.ndarray:
    """All codewords as uint8 [C, N], by testing every word."""
    assert n_vars <= 20
    words = np.arange(1 << n_vars, dtype=np.int64)
    good = np.ones(words.size, dtype=bool)
    for r in rows:
        par = np.zeros(words.size, dtype=np.int64)
        for n in r:
            par ^= (words >> int(n)) & 1
        good &= par == 0
    cw = words[good]
    return ((cw[:, None] >> np.arange(n_vars)[None, :]) & 1).astype(np.uint8)


def correlations(cw: np.ndarray, q0: np.ndarray) -> np.ndarray:
    """corr[f, c] = sum_n (1 - 2 cw[c, n]) q0[f, n]."""
    s = 1.0 - 2.0 * cw.astype(np.float64)
    return np.atleast_2d(q0).astype(np.float64) @ s.T


def ml_decode(cw: np.ndarray, q0: np.ndarray):
    """Returns (ml codewords [F, N], best corr [F], tie flag [F])."""
    corr = correlations(cw, q0)
    best = corr.max(axis=1)
    tie = (corr == best[:, None]).sum(axis=1) > 1
    return cw[corr.argmax(axis=1)], best, tie


def max_marginals(cw: np.ndarray, q0: np.ndarray) -> np.ndarray:
    """Z_ml[f, n] = 1/2 (max over codewords with x_n = 0 - max with x_n = 1)."""
    corr = correlations(cw, q0)                        # F x C
    out = np.zeros((corr.shape[0], cw.shape[1]))
    for n in range(cw.shape[1]):
        z0 = corr[:, cw[:, n] == 0].max(axis=1)
        z1 = corr[:, cw[:, n] == 1].max(axis=1) if np.any(cw[:, n] == 1) else np.full(corr.shape[0], -np.inf)
        out[:, n] = 0.5 * (z0 - z1)
    return out


def app_llr(cw: np.ndarray, q0: np.ndarray) -> np.ndarray:
    """Exact a-posteriori LLRs for channel LLRs q0 (uniform prior over the
    codewords): ln sum over codewords with x_n = 0 of exp(corr/2) minus the same
    over x_n = 1, corr = sum_i (1 - 2 c_i) q0_i (the sum-product decoder's target,
    exact on cycle-free Tanner graphs)."""
    corr = 0.5 * correlations(cw, np.asarray(q0, dtype=float))       # F x C
    out = np.zeros((corr.shape[0], cw.shape[1]))
    for n in range(cw.shape[1]):
        a, b = corr[:, cw[:, n] == 0], corr[:, cw[:, n] == 1]
        la = a.max(axis=1) + np.log(np.exp(a - a.max(axis=1, keepdims=True)).sum(axis=1))
        if b.shape[1] == 0:
            out[:, n] = np.inf
            continue
        lb = b.max(axis=1) + np.log(np.exp(b - b.max(axis=1, keepdims=True)).sum(axis=1))
        out[:, n] = la - lb
    return out
