"""GF(2) encoding for seeded codewords (inputs only; no decoder arithmetic).

The reduced row-echelon form of H gives pivot (parity) columns and free
(information) columns; a codeword is any choice of free bits with the pivot
bits solved from the echelon rows.  Staircase codes are encoded directly by
back-substitution along the dual diagonal.
"""
from __future__ import annotations

import numpy as np

from .codes import Code


def _pack_rows(H: np.ndarray) -> np.ndarray:
    return np.packbits(H, axis=1, bitorder="little").view(np.uint8)


def rref_gf2(H: np.ndarray):
    """Row-reduce a dense 0/1 matrix over GF(2).  Returns (R, pivots) where R has
    ``len(pivots)`` rows in reduced echelon form and pivots[i] is row i's pivot column."""
    M, N = H.shape
    words = (N + 63) // 64
    P = np.zeros((M, words * 8), dtype=np.uint8)
    P[:, : (N + 7) // 8] = _pack_rows(H)
    A = P.view(np.uint64).copy()
    pivots = []
    r = 0
    for c in range(N):
        if r == M:
            break
        w, b = divmod(c, 64)
        bit = np.uint64(1) << np.uint64(b)
        col = (A[r:, w] & bit) != 0
        nz = np.nonzero(col)[0]
        if nz.size == 0:
            continue
        p = r + int(nz[0])
        if p != r:
            A[[r, p]] = A[[p, r]]
        hit = (A[:, w] & bit) != 0
        hit[r] = False
        A[hit] ^= A[r]
        pivots.append(c)
        r += 1
    R = np.unpackbits(A[:r].view(np.uint8), axis=1, bitorder="little")[:, :N]
    return R.astype(np.uint8), np.asarray(pivots, dtype=np.int64)


class Encoder:
    """Maps information bits onto codewords of a code (systematic in the free columns)."""

    def __init__(self, code: Code):
        self.code = code
        self.staircase = code.meta.get("family") == "staircase"
        if self.staircase:
            self.K = code.n_vars - code.n_checks
            self.info_cols = np.arange(self.K)
            return
        R, piv = rref_gf2(code.dense())
        free = np.setdiff1d(np.arange(code.n_vars), piv)
        self.pivots = piv
        self.info_cols = free
        self.K = free.size
        self.Rf = R[:, free].astype(np.float32)  # rank x K

    def encode(self, info: np.ndarray) -> np.ndarray:
        """info: uint8 [F, K] -> codewords uint8 [F, N]."""
        info = np.asarray(info, dtype=np.uint8)
        F = info.shape[0]
        N = self.code.n_vars
        cw = np.zeros((F, N), dtype=np.uint8)
        if self.staircase:
            K = self.K
            M = self.code.n_checks
            cw[:, :K] = info
            rp, ci = self.code.row_ptr, self.code.col_idx
            # row i's info part: the first (deg - parity edges) entries
            s = np.zeros((F, M), dtype=np.uint8)
            for i in range(M):
                cols = ci[rp[i]:rp[i + 1]]
                cols = cols[cols < K]
                s[:, i] = np.bitwise_xor.reduce(info[:, cols], axis=1)
            cw[:, K:] = np.bitwise_xor.accumulate(s, axis=1)
            return cw
        cw[:, self.info_cols] = info
        if self.pivots.size:
            par = (info.astype(np.float32) @ self.Rf.T).astype(np.int64) & 1
            cw[:, self.pivots] = par.astype(np.uint8)
        return cw

    def random_codewords(self, n_frames: int, seed: int) -> np.ndarray:
        rng = np.random.Generator(np.random.Philox(key=seed))
        info = rng.integers(0, 2, size=(n_frames, self.K), dtype=np.uint8)
        return self.encode(info)


def syndrome(code: Code, words: np.ndarray) -> np.ndarray:
    """Per-frame count of unsatisfied checks (uint8 words [F, N])."""
    words = np.asarray(words, dtype=np.uint8)
    rp, ci = code.row_ptr, code.col_idx
    deg = np.diff(rp)
    bits = words[:, ci]  # F x E
    assert np.all(deg > 0)
    # segment xor via cumulative sums mod 2
    cs = np.cumsum(bits, axis=1, dtype=np.int64)
    ends = cs[:, rp[1:] - 1]
    starts = np.concatenate([np.zeros((words.shape[0], 1), np.int64), cs[:, rp[1:-1] - 1]], axis=1)
    par = ((ends - starts) & 1).astype(np.uint8)
    return par.sum(axis=1)
