"""CPU oracle for single-scan min-sum LDPC decoding -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The decoder itself lives in C (``ldpc_oracle.c``),
written from Section III (Eqs. (1), (2)), Section IV (Eq. (3)) and Section V
(Eqs. (4), (5)) of Huang, "Single-Scan Min-Sum Algorithms for Fast Decoding of
LDPC Codes".  This wrapper only marshals numpy arrays; it shares no code with
the CUDA path.  ``brute_force`` holds the exhaustive ML / max-marginal decoders
used to pin the oracle on codes with N <= 20.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, "ldpc_oracle.c")]

TWO_SCAN, SS_FIXED, SS_1BIT = 0, 1, 2
PLAIN, OFFSET, NORMALIZED, SUM_PRODUCT = 0, 1, 2, 3
FORMS = {"two_scan": TWO_SCAN, "ss_fixed": SS_FIXED, "ss_1bit": SS_1BIT}
RULES = {"plain": PLAIN, "offset": OFFSET, "normalized": NORMALIZED, "sum_product": SUM_PRODUCT}
SPA_SAT = 30.0  # |input| saturation of the sum-product check rule


def build(force: bool = False) -> str:
    """Compile the oracle with gcc -O2 (no SIMD intrinsics) into oracle/liboracle.so."""
    newest = max(os.path.getmtime(p) for p in _SRC + [os.path.join(_HERE, "ldpc_oracle.h")])
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp] + _SRC + ["-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Code(ctypes.Structure):
    _fields_ = [("n_vars", ctypes.c_int32), ("n_checks", ctypes.c_int32),
                ("row_ptr", ctypes.POINTER(ctypes.c_int32)),
                ("col_idx", ctypes.POINTER(ctypes.c_int32))]


class _IParams(ctypes.Structure):
    _fields_ = [("rule", ctypes.c_int32), ("offset", ctypes.c_int32),
                ("norm_num", ctypes.c_int32), ("norm_shift", ctypes.c_int32),
                ("msg_sat", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("early_stop", ctypes.c_int32), ("post_sat", ctypes.c_int32)]


class _DParams(ctypes.Structure):
    _fields_ = [("rule", ctypes.c_int32), ("offset", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("early_stop", ctypes.c_int32),
                ("beta_tab", ctypes.POINTER(ctypes.c_double))]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.orc_decode_int.argtypes = [P, P, ctypes.c_int32, P, ctypes.c_int32, P, P, P, P, P, P,
                                        ctypes.c_int32]
        _lib.orc_decode_int.restype = ctypes.c_int
        _lib.orc_decode_f64.argtypes = [P, P, ctypes.c_int32, P, ctypes.c_int32, P, P, P, P, P,
                                        ctypes.c_int32]
        _lib.orc_decode_f64.restype = ctypes.c_int
        _lib.orc_decode_f64_margin.argtypes = [P, P, ctypes.c_int32, P, ctypes.c_int32, P, P, P, P, P, P,
                                               ctypes.c_int32]
        _lib.orc_decode_f64_margin.restype = ctypes.c_int
        _lib.orc_default_threads.restype = ctypes.c_int32
    return _lib


def default_threads() -> int:
    return int(_load().orc_default_threads())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Result(dict):
    """bits [F,N] uint8, iters [F], ok [F], z [F,N], optional l [F,E], state [F,M,4]."""
    __getattr__ = dict.__getitem__


def _code_struct(row_ptr, col_idx, n_vars):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    c = _Code(int(n_vars), int(rp.size - 1), rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
              ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return c, (rp, ci)


def decode_int(code, q0, *, form="ss_1bit", rule="plain", offset=0, norm_num=3, norm_shift=2,
               msg_sat=127, max_iter=20, early_stop=1, post_sat=0, want_l=False, want_state=False,
               threads=0) -> Result:
    """Integer min-sum decode of q0 (int [F, N]) with the given form and rule.
    ``code`` is any object with n_vars, row_ptr, col_idx.  ``post_sat`` > 0
    stores the posterior saturated to [-post_sat, post_sat] after every
    iteration (single-scan forms; 127: an int8 posterior)."""
    lib = _load()
    q = np.ascontiguousarray(np.atleast_2d(q0), dtype=np.int32)
    F, N = q.shape
    assert N == code.n_vars
    c, keep = _code_struct(code.row_ptr, code.col_idx, code.n_vars)
    E = int(keep[0][-1])
    M = keep[0].size - 1
    p = _IParams(RULES[rule], int(offset), int(norm_num), int(norm_shift), int(msg_sat),
                 int(max_iter), int(early_stop), int(post_sat))
    bits = np.zeros((F, N), np.uint8)
    iters = np.zeros(F, np.int32)
    ok = np.zeros(F, np.uint8)
    z = np.zeros((F, N), np.int32)
    l_out = np.zeros((F, E), np.int32) if want_l else None
    st = np.zeros((F, M, 4), np.int32) if want_state else None
    rc = lib.orc_decode_int(ctypes.byref(c), ctypes.byref(p), FORMS[form], _ptr(q), F, _ptr(bits),
                            _ptr(iters), _ptr(ok), _ptr(z), _ptr(l_out), _ptr(st), int(threads))
    if rc != 0:
        raise ValueError("orc_decode_int rejected its arguments")
    r = Result(bits=bits, iters=iters, ok=ok, z=z)
    if want_l:
        r["l"] = l_out
    if want_state:
        r["state"] = st
    return r


def decode_layered_int(code, q0, layer, *, rule="plain", offset=0, norm_num=3, norm_shift=2, msg_sat=127,
                       max_iter=20, early_stop=1, want_l=False, threads=0) -> Result:
    """The single scan of Eq. (3) in a layered schedule: ``layer[m]`` is the
    layer of check m (checks of one layer share no variable); layers run in
    increasing order and update the posteriors in place."""
    lib = _load()
    if not hasattr(lib, "_lay_ready"):
        P = ctypes.c_void_p
        lib.orc_decode_layered_int.argtypes = [P, P, P, ctypes.c_int32, P, ctypes.c_int32, P, P, P, P, P,
                                               ctypes.c_int32]
        lib.orc_decode_layered_int.restype = ctypes.c_int
        lib._lay_ready = True
    q = np.ascontiguousarray(np.atleast_2d(q0), dtype=np.int32)
    F, N = q.shape
    assert N == code.n_vars
    c, keep = _code_struct(code.row_ptr, code.col_idx, code.n_vars)
    E = int(keep[0][-1])
    lay = np.ascontiguousarray(layer, dtype=np.int32)
    p = _IParams(RULES[rule], int(offset), int(norm_num), int(norm_shift), int(msg_sat),
                 int(max_iter), int(early_stop), 0)
    bits = np.zeros((F, N), np.uint8)
    iters = np.zeros(F, np.int32)
    ok = np.zeros(F, np.uint8)
    z = np.zeros((F, N), np.int32)
    l_out = np.zeros((F, E), np.int32) if want_l else None
    rc = lib.orc_decode_layered_int(ctypes.byref(c), ctypes.byref(p), _ptr(lay), int(lay.max()) + 1 if lay.size else 1,
                                    _ptr(q), F, _ptr(bits), _ptr(iters), _ptr(ok), _ptr(z), _ptr(l_out),
                                    int(threads))
    if rc != 0:
        raise ValueError("orc_decode_layered_int rejected its arguments (are the layers column-disjoint?)")
    r = Result(bits=bits, iters=iters, ok=ok, z=z)
    if want_l:
        r["l"] = l_out
    return r


def decode_f64(code, q0, *, form="ss_1bit", rule="normalized", offset=0.0, lam=0.75,
               max_iter=50, early_stop=1, beta_tab=None, want_l=False, want_margin=False,
               threads=0) -> Result:
    """Double-precision min-sum decode of q0 (float [F, N]).  ``beta_tab``:
    optional [max_iter, M] per-iteration, per-check offsets (rule must be 'offset').
    ``want_margin`` adds ``margin`` [F]: the frame's smallest |Z^(k)_n| over all
    iterations, its distance to the decision rule."""
    lib = _load()
    q = np.ascontiguousarray(np.atleast_2d(q0), dtype=np.float64)
    F, N = q.shape
    assert N == code.n_vars
    c, keep = _code_struct(code.row_ptr, code.col_idx, code.n_vars)
    E = int(keep[0][-1])
    bt = None
    if beta_tab is not None:
        bt = np.ascontiguousarray(beta_tab, dtype=np.float64)
        assert bt.shape == (max_iter, keep[0].size - 1) and rule == "offset"
    p = _DParams(RULES[rule], float(offset), float(lam), int(max_iter), int(early_stop),
                 bt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if bt is not None else None)
    bits = np.zeros((F, N), np.uint8)
    iters = np.zeros(F, np.int32)
    ok = np.zeros(F, np.uint8)
    z = np.zeros((F, N), np.float64)
    l_out = np.zeros((F, E), np.float64) if want_l else None
    mg = np.zeros(F, np.float64) if want_margin else None
    rc = lib.orc_decode_f64_margin(ctypes.byref(c), ctypes.byref(p), FORMS[form], _ptr(q), F, _ptr(bits),
                                   _ptr(iters), _ptr(ok), _ptr(z), _ptr(l_out), _ptr(mg), int(threads))
    if rc != 0:
        raise ValueError("orc_decode_f64 rejected its arguments")
    r = Result(bits=bits, iters=iters, ok=ok, z=z)
    if want_l:
        r["l"] = l_out
    if want_margin:
        r["margin"] = mg
    return r


def learned_grad(code, q0, beta_tab, *, targets=None, threads=0):
    """FP64 loss (sum over frames and bits of the BCE terms) and its gradient
    w.r.t. beta_tab [K, M] for the learned offset decoder; also each frame's
    distance ``gap`` to the nearest non-differentiable point."""
    lib = _load()
    if not hasattr(lib, "_lg_ready"):
        P = ctypes.c_void_p
        lib.orc_learned_grad_f64.argtypes = [P, ctypes.c_int32, P, P, P, ctypes.c_int32, P, P, P, ctypes.c_int32]
        lib.orc_learned_grad_f64.restype = ctypes.c_int
        lib._lg_ready = True
    q = np.ascontiguousarray(np.atleast_2d(q0), dtype=np.float64)
    F, N = q.shape
    bt = np.ascontiguousarray(beta_tab, dtype=np.float64)
    K, M = bt.shape
    c, keep = _code_struct(code.row_ptr, code.col_idx, code.n_vars)
    assert keep[0].size - 1 == M and N == code.n_vars
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.uint8)
    loss = np.zeros(1, np.float64)
    db = np.zeros((K, M), np.float64)
    gap = np.zeros(F, np.float64)
    rc = lib.orc_learned_grad_f64(ctypes.byref(c), K, _ptr(bt), _ptr(q), _ptr(tg), F, _ptr(loss), _ptr(db),
                                  _ptr(gap), int(threads))
    if rc != 0:
        raise ValueError("orc_learned_grad_f64 rejected its arguments")
    return float(loss[0]), db, gap
