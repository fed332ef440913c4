"""Named synthetic workloads shaped like the paper's test codes (Section I names
DTMB quasi-cyclic irregular codes, DVB-S2 irregular codes and MacKay regular
codes; none of their tables are available, so seeded stand-ins are built).

Each workload fixes the code, channel (Eb/N0, quantization step ``delta`` and
channel saturation ``qc``), decoder settings and batch size.  Decoder settings
are plain dicts of the C-ABI ``ldpc_decode_params`` field names.
"""
from __future__ import annotations

import dataclasses
import functools

import numpy as np

from . import codes as _codes
from .channel import awgn_llr, quantize
from .encode import Encoder


@dataclasses.dataclass
class Workload:
    name: str
    code: _codes.Code
    ebn0_db: float
    delta: float          # LLR quantization step (int paths)
    qc: int               # channel saturation (int paths)
    params: dict          # decoder settings (C-ABI field names)
    n_frames: int
    codewords: np.ndarray | None = None
    llr: np.ndarray | None = None      # float64 [F, N] channel LLRs
    q0: np.ndarray | None = None       # int8 [F, N] quantized LLRs

    @property
    def K(self) -> int:
        return self.code.n_info


@functools.lru_cache(maxsize=None)
def _code(kind: str, n: int, seed: int) -> _codes.Code:
    if kind == "reg36":
        return _codes.regular_code(n, 3, 6, seed)
    if kind == "qc":
        Z = n // 59
        return _codes.qc_code(seed, Z=Z)
    if kind == "irr":
        return _codes.staircase_code(n, seed)
    raise KeyError(kind)


# name -> (code kind, N, code seed, Eb/N0, delta, qc, params, batch)
WORKLOADS = {
    # (3,6)-regular N=1008, 6-bit LLRs and messages, offset 1, 20 iterations.
    "reg36_n1008": ("reg36", 1008, 11, 2.0, 0.25, 31,
                    dict(dtype="int8", rule="offset", offset=1, msg_sat=31,
                         max_iter=20, early_stop=1), 1000),
    # quasi-cyclic 24x59 base, Z=127 (N=7493), int8, offset 2 LSB, 30 iterations.
    "qc_n7493": ("qc", 7493, 21, 2.5, 0.125, 127,
                 dict(dtype="int8", rule="offset", offset=2, msg_sat=127,
                      max_iter=30, early_stop=1), 4096),
    # irregular staircase N=64800, rate 1/2, normalized 0.75, 50 iterations.
    "irr_n64800": ("irr", 64800, 31, 1.0, 0.125, 127,
                   dict(dtype="int8", rule="normalized", norm_num=3, norm_shift=2,
                        norm=0.75, msg_sat=127, max_iter=50, early_stop=1), 1024),
}


def make_workload(name: str, n_frames: int | None = None, ebn0_db: float | None = None,
                  frame_seed: int = 1, zero_codeword: bool = False, with_llr: bool = True,
                  code: _codes.Code | None = None) -> Workload:
    kind, n, cseed, eb, delta, qc, params, batch = WORKLOADS[name]
    c = code if code is not None else _code(kind, n, cseed)
    F = batch if n_frames is None else n_frames
    eb = eb if ebn0_db is None else ebn0_db
    w = Workload(name, c, eb, delta, qc, dict(params), F)
    if not with_llr:
        return w
    if zero_codeword:
        cw = np.zeros((F, c.n_vars), dtype=np.uint8)
    else:
        cw = _encoder(c).random_codewords(F, seed=frame_seed * 7919 + 1)
    rate = c.n_info / c.n_vars
    llr = awgn_llr(cw, eb, rate, seed=frame_seed * 104729 + 3)
    w.codewords = cw
    w.llr = llr
    w.q0 = quantize(llr, delta, qc)
    return w


# The uneven eight-code batch decoded in one launch: three (3,6)-regular codes,
# two quasi-cyclic 24x59 codes (Z = 61, 127) and three staircase codes, each
# with its family's channel quantization and rule, 30 iterations.
# (kind, N, code seed, Eb/N0, delta, qc, params)
_REG = dict(dtype="int8", rule="offset", offset=1, msg_sat=31, max_iter=30, early_stop=1)
_QC = dict(dtype="int8", rule="offset", offset=2, msg_sat=127, max_iter=30, early_stop=1)
_IRR = dict(dtype="int8", rule="normalized", norm_num=3, norm_shift=2, norm=0.75, msg_sat=127, max_iter=30,
            early_stop=1)
MULTI8 = (("reg36", 1008, 11, 2.0, 0.25, 31, _REG),
          ("reg36", 2016, 12, 2.0, 0.25, 31, _REG),
          ("reg36", 4032, 13, 2.0, 0.25, 31, _REG),
          ("qc", 3599, 22, 2.5, 0.125, 127, _QC),
          ("qc", 7493, 21, 2.5, 0.125, 127, _QC),
          ("irr", 16200, 32, 2.0, 0.125, 127, _IRR),
          ("irr", 32400, 33, 2.0, 0.125, 127, _IRR),
          ("irr", 64800, 31, 2.0, 0.125, 127, _IRR))


def multi8_frame_counts(mean_frames: int = 512, seed: int = 4) -> list:
    """Frames per code of the eight-code batch: Poisson(mean_frames), seeded."""
    return [int(x) for x in np.random.default_rng(seed).poisson(mean_frames, size=len(MULTI8))]


def make_multi_workload(frames=None, mean_frames: int = 512, seed: int = 4, frame_seed: int = 1,
                        zero_codeword: bool = False, with_llr: bool = True, codes=None) -> list:
    """The eight-code batch as a list of Workloads (one per code).  ``frames``:
    explicit frame counts (default Poisson(mean_frames)); ``codes``: indices
    into MULTI8 to keep."""
    counts = multi8_frame_counts(mean_frames, seed) if frames is None else list(frames)
    out = []
    for i, (kind, n, cseed, eb, delta, qc, params) in enumerate(MULTI8):
        if codes is not None and i not in codes:
            continue
        c = _code(kind, n, cseed)
        F = counts[i]
        w = Workload(f"multi8/{kind}_n{n}", c, eb, delta, qc, dict(params), F)
        if with_llr:
            cw = (np.zeros((F, c.n_vars), dtype=np.uint8) if zero_codeword
                  else _encoder(c).random_codewords(F, seed=(frame_seed * 7919 + 1) * 31 + i))
            llr = awgn_llr(cw, eb, c.n_info / c.n_vars, seed=(frame_seed * 104729 + 3) * 31 + i)
            w.codewords, w.llr, w.q0 = cw, llr, quantize(llr, delta, qc)
        out.append(w)
    return out


_enc_cache: dict = {}


def _encoder(c: _codes.Code) -> Encoder:
    key = id(c)
    if key not in _enc_cache:
        _enc_cache[key] = Encoder(c)
    return _enc_cache[key]
