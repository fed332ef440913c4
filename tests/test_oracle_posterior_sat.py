"""Pins of the oracle's 8-bit posterior (the single scan with Z_n stored in b
bits, the storage Section IV's cost argument counts for messages, applied to
the posterior): Z^(k)_n = clamp(Z^(0)_n + sum_m L^(k)_mn, -127, 127) after
every iteration, and the next iteration reads the clamped value.

* hand-worked two-check chains (tests/golden/posterior_sat8_chain.json), one
  clamped from below and one from above, for the per-edge and the Section V
  form;
* invariants: |Z| <= 127 throughout; a clamp wider than every reachable
  posterior gives the exact decode; the two-scan and layered decoders, which
  keep no stored Z_n, reject it;
* mutants of the oracle built on the CPU from its own source (clamp at 126,
  upper bound only, no clamp inside the iterations): each must fail the pins.
"""
import ctypes
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_cs_0609090_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "posterior_sat8_chain.json")))


def _chain():
    return I.from_rows(GOLD["code"]["n_vars"], GOLD["code"]["rows"])


def chain_failures(orc) -> list:
    bad = []
    code = _chain()
    for ci, case in enumerate(GOLD["cases"]):
        q = np.array([case["q0"]], dtype=np.int32)
        for form in ("ss_fixed", "ss_1bit"):
            for key, ps in (("exact", 0), ("sat8", GOLD["post_sat"])):
                exp = case[key]
                for k in (1, 2):
                    r = orc.decode_int(code, q, form=form, rule="plain", msg_sat=GOLD["msg_sat"], max_iter=k,
                                       early_stop=0, post_sat=ps, want_l=True)
                    if r.z[0].tolist() != exp[f"Z{k}"] or r.l[0].tolist() != exp[f"L{k}"]:
                        bad.append((ci, form, key, k, r.z[0].tolist(), r.l[0].tolist()))
                if key == "sat8":
                    r = orc.decode_int(code, q, form=form, rule="plain", msg_sat=GOLD["msg_sat"], max_iter=2,
                                       early_stop=0, post_sat=ps)
                    if r.bits[0].tolist() != exp["bits2"] or int(r.ok[0]) != exp["ok2"]:
                        bad.append((ci, form, "decisions"))
    return bad


def invariant_failures(orc) -> list:
    bad = []
    w = I.make_workload("reg36_n1008", n_frames=24, ebn0_db=1.5)
    q = (w.q0.astype(np.int32) * 4).clip(-127, 127)  # large channel values: posteriors pass 127
    for form in ("ss_fixed", "ss_1bit"):
        for k in (1, 3, 8):
            r = orc.decode_int(w.code, q, form=form, rule="offset", offset=1, msg_sat=127, max_iter=k,
                               early_stop=0, post_sat=127)
            e = orc.decode_int(w.code, q, form=form, rule="offset", offset=1, msg_sat=127, max_iter=k,
                               early_stop=0)
            if np.abs(r.z).max() > 127:
                bad.append((form, k, "bound"))
            if k == 1 and not np.array_equal(r.z, e.z.clip(-127, 127)):
                bad.append((form, k, "first iteration"))  # Z^(0) is the same: only the output clamps
            if k == 8 and np.array_equal(r.z, e.z.clip(-127, 127)):
                bad.append((form, k, "clamp has no effect"))
        wide = orc.decode_int(w.code, q, form=form, rule="offset", offset=1, msg_sat=127, max_iter=8,
                              early_stop=1, post_sat=127 + 3 * 127)
        e = orc.decode_int(w.code, q, form=form, rule="offset", offset=1, msg_sat=127, max_iter=8, early_stop=1)
        for key in ("z", "bits", "iters", "ok"):
            if not np.array_equal(wide[key], e[key]):
                bad.append((form, "wide clamp", key))
    return bad


def test_chain_traces(oracle_lib):
    assert chain_failures(oracle) == []


def test_invariants(oracle_lib):
    assert invariant_failures(oracle) == []


def test_forms_without_a_stored_posterior_reject_it(oracle_lib):
    code = _chain()
    q = np.array([GOLD["cases"][0]["q0"]], dtype=np.int32)
    with pytest.raises(ValueError):
        oracle.decode_int(code, q, form="two_scan", post_sat=127)


_CALL = "if (form != ORC_TWO_SCAN) sat_post(p, Z, N);"
_BODY = "Z[n] = Z[n] > p->post_sat ? p->post_sat : (Z[n] < -p->post_sat ? -p->post_sat : Z[n]);"
_MUTANTS = {
    "clamp at 126": [(_BODY, "Z[n] = Z[n] > p->post_sat - 1 ? p->post_sat - 1 : "
                             "(Z[n] < -(p->post_sat - 1) ? -(p->post_sat - 1) : Z[n]);")],
    "upper bound only": [(_BODY, "Z[n] = Z[n] > p->post_sat ? p->post_sat : Z[n];")],
    "no clamp in the iterations": [(_CALL, "")],
}


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_pins_reject_posterior_mutants(oracle_lib, tmp_path, monkeypatch, name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = open(os.path.join(os.path.dirname(oracle.__file__), "ldpc_oracle.c")).read()
    for old, new in _MUTANTS[name]:
        assert src.count(old) == 1, f"mutation site not found: {old!r}"
        src = src.replace(old, new)
    d = tmp_path / "mut"
    d.mkdir()
    (d / "ldpc_oracle.c").write_text(src)
    shutil.copy(os.path.join(os.path.dirname(oracle.__file__), "ldpc_oracle.h"), d / "ldpc_oracle.h")
    so = str(d / "libmut.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", so,
                           str(d / "ldpc_oracle.c"), "-lm"])
    lib = ctypes.CDLL(so)
    P = ctypes.c_void_p
    lib.orc_decode_int.argtypes = [P, P, ctypes.c_int32, P, ctypes.c_int32, P, P, P, P, P, P, ctypes.c_int32]
    lib.orc_decode_int.restype = ctypes.c_int
    monkeypatch.setattr(oracle, "_lib", lib)
    assert chain_failures(oracle) + invariant_failures(oracle), f"the pins accept the mutant '{name}'"
