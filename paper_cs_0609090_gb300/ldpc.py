"""Thin Python binding over the C ABI in include/ldpc_gb300.h.

The functions keep the C names and only marshal arguments: torch tensors are
passed as ``data_ptr()`` and the current CUDA stream as its handle.  Every step
of decoding runs in the CUDA kernels of libldpc_gb300.so; if that library is
missing, importing this module raises ImportError (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libldpc_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
_lib = ctypes.CDLL(LIB_PATH)

LDPC_OK, LDPC_ERR_INVALID_ARG, LDPC_ERR_UNSUPPORTED, LDPC_ERR_CUDA, LDPC_ERR_OOM, LDPC_ERR_TIMEOUT = range(6)
LDPC_DTYPE_INT8, LDPC_DTYPE_F32 = 0, 1
LDPC_FORM_SS_FIXED, LDPC_FORM_SS_1BIT, LDPC_FORM_TWO_SCAN, LDPC_FORM_TWO_SCAN_1BIT = 0, 1, 2, 3
LDPC_RULE_PLAIN, LDPC_RULE_OFFSET, LDPC_RULE_NORMALIZED, LDPC_RULE_SUM_PRODUCT = 0, 1, 2, 3

DTYPES = {"int8": LDPC_DTYPE_INT8, "f32": LDPC_DTYPE_F32, "float32": LDPC_DTYPE_F32}
FORMS = {"ss_fixed": LDPC_FORM_SS_FIXED, "ss_1bit": LDPC_FORM_SS_1BIT, "two_scan": LDPC_FORM_TWO_SCAN,
         "two_scan_1bit": LDPC_FORM_TWO_SCAN_1BIT}
RULES = {"plain": LDPC_RULE_PLAIN, "offset": LDPC_RULE_OFFSET, "normalized": LDPC_RULE_NORMALIZED,
         "sum_product": LDPC_RULE_SUM_PRODUCT}
(LDPC_KERNEL_AUTO, LDPC_KERNEL_ONCHIP_INT, LDPC_KERNEL_ONCHIP_HALF, LDPC_KERNEL_STREAM, LDPC_KERNEL_CLUSTER,
 LDPC_KERNEL_PERSISTENT, LDPC_KERNEL_PINGPONG) = range(7)
LDPC_SCHEDULE_FLOODING, LDPC_SCHEDULE_LAYERED = 0, 1
SCHEDULES = {"flooding": LDPC_SCHEDULE_FLOODING, "layered": LDPC_SCHEDULE_LAYERED}
LDPC_POSTERIOR_EXACT, LDPC_POSTERIOR_SAT8 = 0, 1
POSTERIORS = {"exact": LDPC_POSTERIOR_EXACT, "sat8": LDPC_POSTERIOR_SAT8}
KERNELS = {"auto": LDPC_KERNEL_AUTO, "onchip_int": LDPC_KERNEL_ONCHIP_INT, "onchip_half": LDPC_KERNEL_ONCHIP_HALF,
           "stream": LDPC_KERNEL_STREAM, "cluster": LDPC_KERNEL_CLUSTER, "persistent": LDPC_KERNEL_PERSISTENT,
           "pingpong": LDPC_KERNEL_PINGPONG}

# Every symbol include/ldpc_gb300.h declares.
EXPORTS = ("ldpc_code_create", "ldpc_code_destroy", "ldpc_code_info", "ldpc_workspace_size",
           "ldpc_decode_batch", "ldpc_decode_batch_noalloc", "ldpc_code_degree_classes",
           "ldpc_learned_workspace_size", "ldpc_learned_forward", "ldpc_learned_loss", "ldpc_learned_backward",
           "ldpc_adam_step", "ldpc_awgn_llr_f32", "ldpc_quantize_llr", "ldpc_multi_create", "ldpc_multi_destroy",
           "ldpc_multi_workspace_size", "ldpc_multi_decode", "ldpc_multi_autotune", "ldpc_multi_info",
           "ldpc_code_layers", "ldpc_code_set_layers", "ldpc_wait_selftest", "ldpc_kernel_choice",
           "ldpc_qc_expand", "ldpc_code_create_qc", "ldpc_last_error")
NOALLOC_SCRATCH_BYTES = 48 * 1024 * 1024


class LdpcError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: status {status}: {ldpc_last_error()}")


class ldpc_decode_params(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("form", ctypes.c_int32), ("rule", ctypes.c_int32),
                ("offset", ctypes.c_int32), ("norm_num", ctypes.c_int32), ("norm_shift", ctypes.c_int32),
                ("offset_f32", ctypes.c_float), ("norm_f32", ctypes.c_float),
                ("msg_sat", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("early_stop", ctypes.c_int32), ("kernel", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("posterior", ctypes.c_int32)]


class ldpc_qc_desc(ctypes.Structure):
    _fields_ = [("base_rows", ctypes.c_int32), ("base_cols", ctypes.c_int32), ("lift", ctypes.c_int32),
                ("shift", ctypes.c_void_p)]


class ldpc_multi_job(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("params", ldpc_decode_params), ("llr", ctypes.c_void_p),
                ("n_frames", ctypes.c_int32), ("hard_bits", ctypes.c_void_p), ("iters_used", ctypes.c_void_p),
                ("syndrome_ok", ctypes.c_void_p), ("llr_out", ctypes.c_void_p)]


class ldpc_multi_tuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("team_threads", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("queue", ctypes.c_int32), ("large", ctypes.c_int32), ("overlap", ctypes.c_int32),
                ("stream_warps", ctypes.c_int32)]


_P = ctypes.c_void_p
_lib.ldpc_code_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_int]
_lib.ldpc_code_destroy.argtypes = [_P]
_lib.ldpc_code_info.argtypes = [_P, _P, _P, _P, _P, _P]
_lib.ldpc_workspace_size.argtypes = [_P, ctypes.POINTER(ldpc_decode_params), ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_size_t)]
_lib.ldpc_decode_batch.argtypes = [_P, ctypes.POINTER(ldpc_decode_params), _P, ctypes.c_int32, _P, _P, _P,
                                   _P, _P, ctypes.c_size_t, _P]
_lib.ldpc_decode_batch_noalloc.argtypes = [_P, ctypes.POINTER(ldpc_decode_params), _P, ctypes.c_int32, _P, _P,
                                           _P, _P, _P]
_lib.ldpc_code_degree_classes.argtypes = [_P, _P, _P]
_lib.ldpc_learned_workspace_size.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
_lib.ldpc_learned_forward.argtypes = [_P, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, _P, ctypes.c_size_t, _P]
_lib.ldpc_learned_loss.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, ctypes.c_size_t,
                                   _P]
_lib.ldpc_learned_backward.argtypes = [_P, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, _P, ctypes.c_size_t, _P]
_lib.ldpc_adam_step.argtypes = [_P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, ctypes.c_float, _P]
_lib.ldpc_awgn_llr_f32.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_float,
                                   ctypes.c_float, ctypes.c_float, _P, _P, _P, _P]
_lib.ldpc_quantize_llr.argtypes = [_P, ctypes.c_int64, ctypes.c_float, ctypes.c_int32, _P, _P]
_lib.ldpc_code_layers.argtypes = [_P, _P, _P]
_lib.ldpc_code_set_layers.argtypes = [_P, ctypes.c_int32, _P]
_lib.ldpc_multi_create.argtypes = [ctypes.POINTER(_P), ctypes.POINTER(ldpc_multi_job), ctypes.c_int32,
                                   ctypes.POINTER(ldpc_multi_tuning)]
_lib.ldpc_multi_destroy.argtypes = [_P]
_lib.ldpc_multi_workspace_size.argtypes = [_P, ctypes.POINTER(ctypes.c_size_t)]
_lib.ldpc_multi_decode.argtypes = [_P, _P, ctypes.c_size_t, _P]
_lib.ldpc_multi_autotune.argtypes = [_P, _P, ctypes.c_size_t, ctypes.c_int32, _P, ctypes.POINTER(ldpc_multi_tuning),
                                     ctypes.POINTER(ctypes.c_float)]
_lib.ldpc_multi_info.argtypes = [_P, ctypes.POINTER(ldpc_multi_tuning), _P, _P, _P, _P, _P]
_lib.ldpc_wait_selftest.argtypes = [ctypes.c_int, ctypes.c_int32]
_lib.ldpc_kernel_choice.argtypes = [_P, ctypes.POINTER(ldpc_decode_params), ctypes.c_int32, _P]
_lib.ldpc_qc_expand.argtypes = [ctypes.POINTER(ldpc_qc_desc), _P, _P, ctypes.c_int64, _P]
_lib.ldpc_code_create_qc.argtypes = [ctypes.POINTER(_P), ctypes.POINTER(ldpc_qc_desc), ctypes.c_int]
_lib.ldpc_last_error.restype = ctypes.c_char_p
for _f in EXPORTS[:-1]:
    getattr(_lib, _f).restype = ctypes.c_int32


def _check(status: int, where: str):
    if status != LDPC_OK:
        raise LdpcError(status, where)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(_P)
    return _P(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    if hasattr(stream, "cuda_stream"):
        return _P(stream.cuda_stream)
    return _P(int(stream))


def ldpc_kernel_choice(code: int, params: ldpc_decode_params, n_frames: int) -> str:
    """Name (a KERNELS key) of the implementation ldpc_decode_batch runs."""
    out = ctypes.c_int32(0)
    _check(_lib.ldpc_kernel_choice(_P(code), ctypes.byref(params), int(n_frames), ctypes.byref(out)),
           "ldpc_kernel_choice")
    return {v: k for k, v in KERNELS.items()}[out.value]


def ldpc_wait_selftest(device: int, max_spins: int) -> int:
    """Status of the persistent decoder's bounded wait run on a counter that
    nothing increments (LDPC_ERR_TIMEOUT is the expected answer)."""
    return int(_lib.ldpc_wait_selftest(int(device), int(max_spins)))


def ldpc_last_error() -> str:
    return (_lib.ldpc_last_error() or b"").decode()


def make_params(dtype="int8", form="ss_1bit", rule="offset", offset=0, norm_num=3, norm_shift=2,
                offset_f32=0.0, norm_f32=0.75, msg_sat=127, max_iter=20, early_stop=1,
                norm=None, kernel="auto", schedule="flooding", posterior="exact", **_ignored) -> ldpc_decode_params:
    """Builds ldpc_decode_params from names ('int8'/'f32', 'ss_fixed'/'ss_1bit'/'two_scan'/'two_scan_1bit',
    'plain'/'offset'/'normalized', 'flooding'/'layered', 'exact'/'sat8').  ``norm`` is an alias for
    norm_f32."""
    if norm is not None:
        norm_f32 = norm
    return ldpc_decode_params(DTYPES[dtype] if isinstance(dtype, str) else dtype,
                              FORMS[form] if isinstance(form, str) else form,
                              RULES[rule] if isinstance(rule, str) else rule,
                              int(offset), int(norm_num), int(norm_shift), float(offset_f32),
                              float(norm_f32), int(msg_sat), int(max_iter), int(early_stop),
                              KERNELS[kernel] if isinstance(kernel, str) else int(kernel),
                              SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule),
                              POSTERIORS[posterior] if isinstance(posterior, str) else int(posterior))


def ldpc_code_create(n_vars: int, n_checks: int, row_ptr, col_idx, device: int = 0) -> int:
    """Returns an opaque handle (int).  row_ptr/col_idx: host int32 arrays."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    h = _P()
    _check(_lib.ldpc_code_create(ctypes.byref(h), int(n_vars), int(n_checks), _ptr(rp), _ptr(ci), int(device)),
           "ldpc_code_create")
    return h.value


def _qc_desc(shifts, lift: int):
    sh = np.ascontiguousarray(shifts, dtype=np.int32)
    assert sh.ndim == 2
    return ldpc_qc_desc(sh.shape[0], sh.shape[1], int(lift), sh.ctypes.data), sh


def ldpc_qc_expand(shifts, lift: int):
    """(row_ptr, col_idx) int32 of the quasi-cyclic code whose base matrix of
    circulant shifts is ``shifts`` [mb, nb] (-1: zero block), lifted by ``lift``.
    Host computation only."""
    d, keep = _qc_desc(shifts, lift)
    e = ctypes.c_int32()
    _check(_lib.ldpc_qc_expand(ctypes.byref(d), None, None, 0, ctypes.byref(e)), "ldpc_qc_expand")
    rp = np.zeros(d.base_rows * d.lift + 1, np.int32)
    ci = np.zeros(max(e.value, 1), np.int32)
    _check(_lib.ldpc_qc_expand(ctypes.byref(d), _ptr(rp), _ptr(ci), int(ci.size), None), "ldpc_qc_expand")
    return rp, ci[:e.value]


def ldpc_code_create_qc(shifts, lift: int, device: int = 0) -> int:
    d, keep = _qc_desc(shifts, lift)
    h = _P()
    _check(_lib.ldpc_code_create_qc(ctypes.byref(h), ctypes.byref(d), int(device)), "ldpc_code_create_qc")
    return h.value


def ldpc_code_destroy(code: int) -> None:
    _check(_lib.ldpc_code_destroy(_P(code)), "ldpc_code_destroy")


def ldpc_code_info(code: int) -> dict:
    vals = [ctypes.c_int32() for _ in range(5)]
    _check(_lib.ldpc_code_info(_P(code), *[ctypes.byref(v) for v in vals]), "ldpc_code_info")
    return dict(zip(("n_vars", "n_checks", "n_edges", "max_row_degree", "max_col_degree"),
                    (v.value for v in vals)))


def ldpc_workspace_size(code: int, params: ldpc_decode_params, n_frames: int) -> int:
    out = ctypes.c_size_t()
    _check(_lib.ldpc_workspace_size(_P(code), ctypes.byref(params), int(n_frames), ctypes.byref(out)),
           "ldpc_workspace_size")
    return out.value


def ldpc_decode_batch(code: int, params: ldpc_decode_params, llr, n_frames: int, hard_bits, iters_used,
                      syndrome_ok, llr_out=None, workspace=None, ws_bytes: int = 0, stream=None) -> None:
    """All tensors are CUDA tensors of the layouts documented in the header."""
    _check(_lib.ldpc_decode_batch(_P(code), ctypes.byref(params), _ptr(llr), int(n_frames), _ptr(hard_bits),
                                  _ptr(iters_used), _ptr(syndrome_ok), _ptr(llr_out), _ptr(workspace),
                                  int(ws_bytes), _stream_handle(stream)), "ldpc_decode_batch")


def ldpc_decode_batch_noalloc(code: int, params: ldpc_decode_params, llr, n_frames: int, hard_bits, iters_used,
                              syndrome_ok, llr_out=None, stream=None) -> None:
    """ldpc_decode_batch for callers that cannot allocate device memory: the
    library's built-in device scratch replaces the workspace (int8 streaming
    decoder; see include/ldpc_gb300.h for the size limit and the rule that calls
    overlapping on the GPU race)."""
    _check(_lib.ldpc_decode_batch_noalloc(_P(code), ctypes.byref(params), _ptr(llr), int(n_frames), _ptr(hard_bits),
                                          _ptr(iters_used), _ptr(syndrome_ok), _ptr(llr_out),
                                          _stream_handle(stream)), "ldpc_decode_batch_noalloc")


def ldpc_code_degree_classes(code: int) -> list:
    n = ctypes.c_int32()
    deg = (ctypes.c_int32 * 32)()
    _check(_lib.ldpc_code_degree_classes(_P(code), ctypes.byref(n), deg), "ldpc_code_degree_classes")
    return [deg[i] for i in range(n.value)]


def ldpc_learned_workspace_size(code: int, n_iters: int, n_frames: int) -> int:
    out = ctypes.c_size_t()
    _check(_lib.ldpc_learned_workspace_size(_P(code), int(n_iters), int(n_frames), ctypes.byref(out)),
           "ldpc_learned_workspace_size")
    return out.value


def ldpc_learned_forward(code: int, n_iters: int, beta, llr, n_frames: int, z_out, workspace, ws_bytes: int,
                         stream=None) -> None:
    _check(_lib.ldpc_learned_forward(_P(code), int(n_iters), _ptr(beta), _ptr(llr), int(n_frames), _ptr(z_out),
                                     _ptr(workspace), int(ws_bytes), _stream_handle(stream)), "ldpc_learned_forward")


def ldpc_learned_loss(code: int, n_iters: int, n_frames: int, target_bits, loss, want_grad: bool, workspace,
                      ws_bytes: int, stream=None) -> None:
    _check(_lib.ldpc_learned_loss(_P(code), int(n_iters), int(n_frames), _ptr(target_bits), _ptr(loss),
                                  int(bool(want_grad)), _ptr(workspace), int(ws_bytes), _stream_handle(stream)),
           "ldpc_learned_loss")


def ldpc_learned_backward(code: int, n_iters: int, beta, dz, n_frames: int, dbeta, workspace, ws_bytes: int,
                          stream=None) -> None:
    _check(_lib.ldpc_learned_backward(_P(code), int(n_iters), _ptr(beta), _ptr(dz), int(n_frames), _ptr(dbeta),
                                      _ptr(workspace), int(ws_bytes), _stream_handle(stream)),
           "ldpc_learned_backward")


def ldpc_adam_step(params, grads, m, v, n: int, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                   eps: float = 1e-8, stream=None) -> None:
    _check(_lib.ldpc_adam_step(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(n), int(step), float(lr),
                               float(beta1), float(beta2), float(eps), _stream_handle(stream)), "ldpc_adam_step")


def ldpc_awgn_llr_f32(n_vars: int, seed: int, first_frame: int, n_frames: int, ebn0_lo_db: float,
                      ebn0_hi_db: float, rate: float, codewords, llr, ebn0_out=None, stream=None) -> None:
    _check(_lib.ldpc_awgn_llr_f32(int(n_vars), int(seed), int(first_frame), int(n_frames), float(ebn0_lo_db),
                                  float(ebn0_hi_db), float(rate), _ptr(codewords), _ptr(llr), _ptr(ebn0_out),
                                  _stream_handle(stream)), "ldpc_awgn_llr_f32")


def ldpc_quantize_llr(llr, n: int, delta: float, qc: int, q, stream=None) -> None:
    _check(_lib.ldpc_quantize_llr(_ptr(llr), int(n), float(delta), int(qc), _ptr(q), _stream_handle(stream)),
           "ldpc_quantize_llr")


def ldpc_code_layers(code: int, n_checks: int):
    """(n_layers, layer_of_check int32 [n_checks]) of the layered schedule."""
    n = ctypes.c_int32()
    lay = np.zeros(n_checks, np.int32)
    _check(_lib.ldpc_code_layers(_P(code), ctypes.byref(n), _ptr(lay)), "ldpc_code_layers")
    return n.value, lay


def ldpc_code_set_layers(code: int, layer_of_check) -> None:
    lay = np.ascontiguousarray(layer_of_check, dtype=np.int32)
    _check(_lib.ldpc_code_set_layers(_P(code), int(lay.max()) + 1, _ptr(lay)), "ldpc_code_set_layers")


def ldpc_multi_create(jobs, tuning: ldpc_multi_tuning | None = None) -> int:
    """jobs: a sequence of ldpc_multi_job.  Returns an opaque plan handle."""
    arr = (ldpc_multi_job * len(jobs))(*jobs)
    h = _P()
    _check(_lib.ldpc_multi_create(ctypes.byref(h), arr, len(jobs), ctypes.byref(tuning) if tuning else None),
           "ldpc_multi_create")
    return h.value


def ldpc_multi_destroy(plan: int) -> None:
    _check(_lib.ldpc_multi_destroy(_P(plan)), "ldpc_multi_destroy")


def ldpc_multi_workspace_size(plan: int) -> int:
    out = ctypes.c_size_t()
    _check(_lib.ldpc_multi_workspace_size(_P(plan), ctypes.byref(out)), "ldpc_multi_workspace_size")
    return out.value


def ldpc_multi_decode(plan: int, workspace, ws_bytes: int, stream=None) -> None:
    _check(_lib.ldpc_multi_decode(_P(plan), _ptr(workspace), int(ws_bytes), _stream_handle(stream)),
           "ldpc_multi_decode")


def ldpc_multi_autotune(plan: int, workspace, ws_bytes: int, reps: int = 3, stream=None):
    """Returns (chosen ldpc_multi_tuning, mean ms of the kept shape)."""
    t = ldpc_multi_tuning()
    ms = ctypes.c_float()
    _check(_lib.ldpc_multi_autotune(_P(plan), _ptr(workspace), int(ws_bytes), int(reps), _stream_handle(stream),
                                    ctypes.byref(t), ctypes.byref(ms)), "ldpc_multi_autotune")
    return t, ms.value


def ldpc_multi_info(plan: int, n_jobs: int) -> dict:
    t = ldpc_multi_tuning()
    grid, cluster, smem = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    is_cl = (ctypes.c_int32 * n_jobs)()
    pairs = (ctypes.c_int32 * n_jobs)()
    _check(_lib.ldpc_multi_info(_P(plan), ctypes.byref(t), ctypes.byref(grid), ctypes.byref(cluster),
                                ctypes.byref(smem), is_cl, pairs), "ldpc_multi_info")
    return {"threads": t.threads, "team_threads": t.team_threads, "cluster": cluster.value, "queue": t.queue,
            "large": t.large, "overlap": t.overlap, "stream_warps": t.stream_warps, "grid": grid.value,
            "smem_bytes": smem.value,
            "job_is_cluster": list(is_cl),
            "job_pairs_per_cta": list(pairs)}


class Code:
    """Owning wrapper of an ldpc_code handle."""

    def __init__(self, n_vars, n_checks, row_ptr, col_idx, device=0):
        self.handle = ldpc_code_create(n_vars, n_checks, row_ptr, col_idx, device)
        self.n_vars, self.n_checks = int(n_vars), int(n_checks)
        self.device = device

    @classmethod
    def from_qc(cls, shifts, lift, device=0):
        """A quasi-cyclic code from its base matrix of circulant shifts (-1: zero
        block) and lift; its layers are the block rows."""
        obj = cls.__new__(cls)
        sh = np.asarray(shifts)
        obj.handle = ldpc_code_create_qc(sh, lift, device)
        obj.n_vars, obj.n_checks = int(sh.shape[1] * lift), int(sh.shape[0] * lift)
        obj.device = device
        return obj

    @classmethod
    def from_inputs(cls, code, device=0):
        return cls(code.n_vars, code.n_checks, code.row_ptr, code.col_idx, device)

    def close(self):
        if getattr(self, "handle", None):
            ldpc_code_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def decode(code: Code, llr, params: ldpc_decode_params, want_llr: bool = False, stream=None,
           workspace=None):
    """Allocates outputs with torch on llr's device and calls ldpc_decode_batch.
    Returns (hard_bits uint8 [F, ceil(N/8)], iters int32 [F], ok uint8 [F], llr_out or None)."""
    import torch
    F, N = llr.shape
    dev = llr.device
    bits = torch.empty((F, (N + 7) // 8), dtype=torch.uint8, device=dev)
    iters = torch.empty(F, dtype=torch.int32, device=dev)
    ok = torch.empty(F, dtype=torch.uint8, device=dev)
    zo = None
    if want_llr:
        zo = torch.empty((F, N), dtype=torch.int16 if params.dtype == LDPC_DTYPE_INT8 else torch.float32,
                         device=dev)
    ws_bytes = ldpc_workspace_size(code.handle, params, F)
    if ws_bytes and workspace is None:
        workspace = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=dev)
    ws_ptr = None
    if ws_bytes:
        base = workspace.data_ptr()
        ws_ptr = _P((base + 255) & ~255)
    _check(_lib.ldpc_decode_batch(_P(code.handle), ctypes.byref(params), _ptr(llr), int(F), _ptr(bits),
                                  _ptr(iters), _ptr(ok), _ptr(zo), ws_ptr, int(ws_bytes),
                                  _stream_handle(stream)), "ldpc_decode_batch")
    return bits, iters, ok, zo


class MultiBatch:
    """A plan over several codes with torch-allocated outputs bound to it:
    ``decode()`` runs every job in one launch (ldpc_multi_decode);
    ``outputs[j]`` = (hard_bits, iters, ok, llr_out or None) of job j."""

    def __init__(self, codes, llrs, params, want_llr: bool = False, tuning: ldpc_multi_tuning | None = None):
        import torch
        self.codes, self.llrs = list(codes), list(llrs)
        self.params = list(params) if isinstance(params, (list, tuple)) else [params] * len(self.codes)
        self.outputs = []
        jobs = []
        for c, q, p in zip(self.codes, self.llrs, self.params):
            F, N = q.shape
            dev = q.device
            bits = torch.zeros((F, (N + 7) // 8), dtype=torch.uint8, device=dev)
            iters = torch.zeros(F, dtype=torch.int32, device=dev)
            ok = torch.zeros(F, dtype=torch.uint8, device=dev)
            zo = torch.zeros((F, N), dtype=torch.int16, device=dev) if want_llr else None
            self.outputs.append((bits, iters, ok, zo))
            jobs.append(ldpc_multi_job(c.handle, p, q.data_ptr(), F, bits.data_ptr(), iters.data_ptr(),
                                       ok.data_ptr(), zo.data_ptr() if zo is not None else None))
        self.handle = ldpc_multi_create(jobs, tuning)
        self.ws_bytes = ldpc_multi_workspace_size(self.handle)
        dev = self.llrs[0].device
        self._ws = torch.empty(max(self.ws_bytes, 1) + 256, dtype=torch.uint8, device=dev)
        self.ws = _P((self._ws.data_ptr() + 255) & ~255) if self.ws_bytes else None

    def decode(self, stream=None) -> None:
        _check(_lib.ldpc_multi_decode(_P(self.handle), self.ws, int(self.ws_bytes), _stream_handle(stream)),
               "ldpc_multi_decode")

    def autotune(self, reps: int = 3, stream=None):
        t = ldpc_multi_tuning()
        ms = ctypes.c_float()
        _check(_lib.ldpc_multi_autotune(_P(self.handle), self.ws, int(self.ws_bytes), int(reps),
                                        _stream_handle(stream), ctypes.byref(t), ctypes.byref(ms)),
               "ldpc_multi_autotune")
        return t, ms.value

    def info(self) -> dict:
        return ldpc_multi_info(self.handle, len(self.codes))

    def close(self):
        if getattr(self, "handle", None):
            ldpc_multi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def unpack_bits(hard_bits: np.ndarray, n_vars: int) -> np.ndarray:
    """[F, ceil(N/8)] packed (bit n at byte n>>3, bit n&7) -> [F, N] uint8."""
    return np.unpackbits(np.asarray(hard_bits, dtype=np.uint8), axis=1, bitorder="little")[:, :n_vars]
