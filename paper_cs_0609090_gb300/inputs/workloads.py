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


_enc_cache: dict = {}


def _encoder(c: _codes.Code) -> Encoder:
    key = id(c)
    if key not in _enc_cache:
        _enc_cache[key] = Encoder(c)
    return _enc_cache[key]
