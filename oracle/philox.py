"""Philox4x32-10 counter-based generator and the AWGN frame construction built
on it -- TEST INFRASTRUCTURE ONLY (the reference for the device generator).

Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC 2011): a 4 x 32-bit counter and a 2 x 32-bit
key; each of the 10 rounds multiplies counter words 0 and 2 by 0xD2511F53 and
0xCD9E8D57 (64-bit products), outputs (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
and adds the Weyl constants 0x9E3779B9 / 0xBB67AE85 to the key.
"""
from __future__ import annotations

import numpy as np

M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """ctr: uint32 [..., 4]; key: (k0, k1).  Returns uint32 [..., 4]."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for _ in range(10):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
        k0 = (k0 + W0) & 0xFFFFFFFF
        k1 = (k1 + W1) & 0xFFFFFFFF
    return np.stack([x.astype(np.uint32) for x in c], axis=-1)


def u01(w: np.ndarray) -> np.ndarray:
    """(0, 1] from the top 24 bits of a word: ((w >> 8) + 1) / 2^24."""
    return ((w >> np.uint32(8)).astype(np.float64) + 1.0) / 16777216.0


def awgn_llr(n_vars: int, seed: int, first_frame: int, n_frames: int, lo: float, hi: float, rate: float,
             codewords=None):
    """Channel LLRs [F, N] and per-frame Eb/N0 [F] with the counter layout of
    ldpc_awgn_llr_f32: counter (g, frame_lo, frame_hi, 0) -> Box-Muller normals
    of variables 4g..4g+3; counter (2^32 - 1, frame_lo, frame_hi, 1) -> Eb/N0."""
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    fr = np.arange(first_frame, first_frame + n_frames, dtype=np.uint64)
    flo, fhi = (fr & MASK).astype(np.uint32), (fr >> np.uint64(32)).astype(np.uint32)
    ce = np.stack([np.full(n_frames, 0xFFFFFFFF, np.uint32), flo, fhi, np.ones(n_frames, np.uint32)], axis=-1)
    ue = philox4x32_10(ce, key)
    eb = lo + (hi - lo) * (u01(ue[:, 0]) - 1.0 / 16777216.0)
    G = (n_vars + 3) // 4
    g = np.arange(G, dtype=np.uint32)
    ctr = np.stack([np.broadcast_to(g[None, :], (n_frames, G)),
                    np.broadcast_to(flo[:, None], (n_frames, G)),
                    np.broadcast_to(fhi[:, None], (n_frames, G)),
                    np.zeros((n_frames, G), np.uint32)], axis=-1)
    w = philox4x32_10(ctr, key)
    r0 = np.sqrt(-2.0 * np.log(u01(w[..., 0])))
    r1 = np.sqrt(-2.0 * np.log(u01(w[..., 2])))
    t0 = 2.0 * np.pi * u01(w[..., 1])
    t1 = 2.0 * np.pi * u01(w[..., 3])
    xi = np.stack([r0 * np.cos(t0), r0 * np.sin(t0), r1 * np.cos(t1), r1 * np.sin(t1)], axis=-1)
    xi = xi.reshape(n_frames, 4 * G)[:, :n_vars]
    s2 = 1.0 / (2.0 * rate * 10.0 ** (eb / 10.0))
    x = np.zeros((n_frames, n_vars)) if codewords is None else np.asarray(codewords, dtype=np.float64)
    y = (1.0 - 2.0 * x) + np.sqrt(s2)[:, None] * xi
    return 2.0 * y / s2[:, None], eb
