"""CPU-only checks of the C-ABI library: it loads, exports every symbol that
include/*.h declares, and rejects malformed requests before touching CUDA."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names |= set(re.findall(r"LDPC_API\s+[\w\s\*]*?\b(ldpc_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def L():
    from paper_cs_0609090_gb300 import ldpc
    return ldpc


def test_library_exports_every_declared_symbol(L):
    declared = _declared_symbols()
    assert declared, "no LDPC_API declarations found"
    lib = ctypes.CDLL(L.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(L.EXPORTS)


def test_struct_layouts_match_the_header(L, tmp_path):
    """sizeof and offsetof of every field of the ABI structs, compiled from the
    header with gcc, equal the binding's ctypes definitions."""
    import subprocess
    structs = {"ldpc_decode_params": L.ldpc_decode_params, "ldpc_multi_job": L.ldpc_multi_job,
               "ldpc_multi_tuning": L.ldpc_multi_tuning, "ldpc_qc_desc": L.ldpc_qc_desc}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ldpc_gb300.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(__file__), "..", "include")
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(out[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)


def _create_raw(L, n_vars, n_checks, rp, ci):
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(rp, np.int32)
    ci = np.ascontiguousarray(ci, np.int32)
    st = L._lib.ldpc_code_create(ctypes.byref(h), n_vars, n_checks, rp.ctypes.data_as(ctypes.c_void_p),
                                 ci.ctypes.data_as(ctypes.c_void_p), 0)
    return st, h


def test_create_rejects_malformed_h(L):
    ok_rp, ok_ci = [0, 4, 8, 12], [0, 1, 3, 4, 0, 2, 3, 5, 1, 2, 3, 6]
    assert _create_raw(L, 7, 3, [1, 4, 8, 12], ok_ci)[0] == L.LDPC_ERR_INVALID_ARG       # row_ptr[0] != 0
    assert "row_ptr[0]" in L.ldpc_last_error()
    assert _create_raw(L, 7, 3, [0, 1, 8, 12], ok_ci)[0] == L.LDPC_ERR_INVALID_ARG       # degree 1
    assert _create_raw(L, 7, 3, ok_rp, [0, 1, 3, 9] + ok_ci[4:])[0] == L.LDPC_ERR_INVALID_ARG  # index
    assert _create_raw(L, 7, 3, ok_rp, [0, 1, 1, 4] + ok_ci[4:])[0] == L.LDPC_ERR_INVALID_ARG  # repeat
    assert "twice" in L.ldpc_last_error()
    assert _create_raw(L, 0, 3, ok_rp, ok_ci)[0] == L.LDPC_ERR_INVALID_ARG
    big = [0, 33]
    assert _create_raw(L, 40, 1, big, list(range(33)))[0] == L.LDPC_ERR_INVALID_ARG     # degree 33
    st = L._lib.ldpc_code_create(None, 7, 3, None, None, 0)
    assert st == L.LDPC_ERR_INVALID_ARG


def test_null_arguments(L):
    p = L.make_params()
    assert L._lib.ldpc_decode_batch(None, ctypes.byref(p), None, 1, None, None, None, None, None, 0,
                                    None) == L.LDPC_ERR_INVALID_ARG
    out = ctypes.c_size_t()
    assert L._lib.ldpc_workspace_size(None, ctypes.byref(p), 1, ctypes.byref(out)) == L.LDPC_ERR_INVALID_ARG
    assert L._lib.ldpc_code_destroy(None) == L.LDPC_OK
    assert L._lib.ldpc_code_info(None, None, None, None, None, None) == L.LDPC_ERR_INVALID_ARG


def test_valid_code_without_gpu_reports_cuda_error(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, h = _create_raw(L, 7, 3, [0, 4, 8, 12], [0, 1, 3, 4, 0, 2, 3, 5, 1, 2, 3, 6])
    assert st in (L.LDPC_ERR_CUDA, L.LDPC_ERR_INVALID_ARG)
    assert h.value is None
    assert L.ldpc_last_error() != ""


def test_unpack_bits_layout(L):
    hb = np.array([[0b00000101, 0b1]], dtype=np.uint8)
    assert L.unpack_bits(hb, 9).tolist() == [[1, 0, 1, 0, 0, 0, 0, 0, 1]]


def test_qc_expand_matches_the_generator(L):
    """ldpc_qc_expand (host code of the library) rebuilds the N=7493 QC code
    from its base matrix of shifts, and small hand-checked cases: one circulant
    row r -> column (r + s) mod z, zero blocks skipped."""
    from paper_cs_0609090_gb300 import inputs as I
    code = I.make_workload("qc_n7493", n_frames=1).code
    rp, ci = L.ldpc_qc_expand(code.meta["shifts"], code.meta["Z"])
    assert np.array_equal(rp, code.row_ptr) and np.array_equal(ci, code.col_idx)
    rp, ci = L.ldpc_qc_expand([[1, -1, 0]], 3)
    assert rp.tolist() == [0, 2, 4, 6]
    assert ci.tolist() == [1, 6, 2, 7, 0, 8]
    rp, ci = L.ldpc_qc_expand([[-1, -1]], 4)
    assert rp.tolist() == [0, 0, 0, 0, 0] and ci.size == 0


def test_qc_expand_rejects_malformed_descriptors(L):
    for shifts, z in (([[3]], 3), ([[-2]], 3), ([[0]], 0)):
        with pytest.raises(L.LdpcError):
            L.ldpc_qc_expand(shifts, z)
    d, keep = L._qc_desc([[0, 1]], 4)
    rp = np.zeros(5, np.int32)
    ci = np.zeros(7, np.int32)  # 8 needed
    st = L._lib.ldpc_qc_expand(ctypes.byref(d), rp.ctypes.data_as(ctypes.c_void_p),
                               ci.ctypes.data_as(ctypes.c_void_p), 7, None)
    assert st == L.LDPC_ERR_INVALID_ARG and "needed" in L.ldpc_last_error()
    assert L._lib.ldpc_qc_expand(None, None, None, 0, None) == L.LDPC_ERR_INVALID_ARG

