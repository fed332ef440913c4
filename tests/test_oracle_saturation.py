"""Pins of the oracle's message saturation (the b-bit message magnitudes of
Section V: every input magnitude |Z_n' - L_mn'| of a check is clamped to Qm
before the minimum of Eq. (1) / Eq. (3), and the normalized / offset rule of
Section III acts on the clamped minimum).

* a hand-worked (7,4) Hamming decode at Qm = 2, plain, offset and normalized
  (tests/golden/hamming74_min_sum.json, sections *_qm2), in which the
  saturation changes messages, posteriors and the Section V state;
* the closed form of one parity check after one iteration with inputs above
  Qm: Z_n = q0_n + prod_{n' != n} sgn(q0_n') g(min(min_{n' != n} |q0_n'|, Qm));
* mutants of the oracle built on the CPU from its own source (clamping to
  Qm - 1 or Qm + 1, no clamp, clamping after the rule): every one of them must
  fail these pins, so the pins see each of those mistakes.
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

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hamming74_min_sum.json")))
FORMS = ["two_scan", "ss_fixed", "ss_1bit"]


def _ham():
    return I.from_rows(GOLD["code"]["n_vars"], GOLD["code"]["rows"])


def _q0():
    return np.array([GOLD["q0"]], dtype=np.int32)


def _rule_g(rule, mag, offset=0, num=3, shift=2):
    if rule == "offset":
        return np.maximum(mag - offset, 0)
    if rule == "normalized":
        return (mag * num) >> shift
    return mag


def hamming_failures(orc) -> list:
    """Differences between the oracle and the hand-worked Qm = 2 traces."""
    bad = []
    code = _ham()
    g = GOLD["plain_qm2"]
    qm = g["msg_sat"]
    for form in FORMS:
        r1 = orc.decode_int(code, _q0(), form=form, rule="plain", msg_sat=qm, max_iter=1, early_stop=0,
                            want_l=True, want_state=(form == "ss_1bit"))
        if r1.z[0].tolist() != g["Z1"]:
            bad.append((form, "plain Z1", r1.z[0].tolist()))
        if r1.l[0].tolist() != sum(g["L1"], []):
            bad.append((form, "plain L1"))
        if r1.bits[0].tolist() != g["k1_bits"] or r1.ok[0] != g["k1_syndrome_ok"]:
            bad.append((form, "plain k1 decisions"))
        if form == "ss_1bit":
            st = r1.state[0]
            for c, key in enumerate(("state1_A", "state1_B", "state1_idx", "state1_signword")):
                if st[:, c].tolist() != g[key]:
                    bad.append((form, key, st[:, c].tolist()))
        r2 = orc.decode_int(code, _q0(), form=form, rule="plain", msg_sat=qm, max_iter=2, early_stop=0,
                            want_l=True, want_state=(form == "ss_1bit"))
        if r2.z[0].tolist() != g["Z2"]:
            bad.append((form, "plain Z2", r2.z[0].tolist()))
        if r2.l[0].tolist() != sum(g["L2"], []):
            bad.append((form, "plain L2"))
        if form == "ss_1bit":
            st = r2.state[0]
            for c, key in enumerate(("state2_A", "state2_B", "state2_idx", "state2_signword")):
                if st[:, c].tolist() != g[key]:
                    bad.append((form, key, st[:, c].tolist()))
        rf = orc.decode_int(code, _q0(), form=form, rule="plain", msg_sat=qm, max_iter=20, early_stop=1)
        if (rf.bits[0].tolist(), int(rf.iters[0]), int(rf.ok[0])) != (g["final_bits"], g["final_iters"],
                                                                      g["final_ok"]):
            bad.append((form, "plain final"))

        o = GOLD["offset1_qm2"]
        r = orc.decode_int(code, _q0(), form=form, rule="offset", offset=1, msg_sat=qm, max_iter=1,
                           early_stop=0, want_l=True, want_state=(form == "ss_1bit"))
        if r.z[0].tolist() != o["Z1"] or r.l[0].tolist() != sum(o["L1"], []):
            bad.append((form, "offset Z1/L1", r.z[0].tolist()))
        if form == "ss_1bit":
            st = r.state[0]
            for c, key in enumerate(("state1_A", "state1_B", "state1_idx", "state1_signword")):
                if st[:, c].tolist() != o[key]:
                    bad.append((form, "offset " + key, st[:, c].tolist()))
        r = orc.decode_int(code, _q0(), form=form, rule="offset", offset=1, msg_sat=qm, max_iter=10)
        if (int(r.iters[0]), int(r.ok[0])) != (o["final_iters"], o["final_ok"]):
            bad.append((form, "offset final"))

        nz = GOLD["normalized_int_3_over_4_qm2"]
        r = orc.decode_int(code, _q0(), form=form, rule="normalized", norm_num=3, norm_shift=2, msg_sat=qm,
                           max_iter=10)
        if r.z[0].tolist() != nz["Z1"] or (int(r.iters[0]), int(r.ok[0])) != (nz["final_iters"],
                                                                              nz["final_ok"]):
            bad.append((form, "normalized Z1", r.z[0].tolist()))
    return bad


def single_check_failures(orc) -> list:
    """Differences from the closed form of one parity check (one iteration)
    with channel values up to 4 Qm in magnitude."""
    bad = []
    rng = np.random.default_rng(11)
    for N, qm in ((5, 3), (7, 17), (9, 31)):
        code = I.from_rows(N, [list(range(N))])
        q0 = rng.integers(-4 * qm, 4 * qm + 1, size=(120, N)).astype(np.int32)
        for rule, kw in (("plain", {}), ("offset", {"offset": 2}), ("normalized", {"norm_num": 3, "norm_shift": 2})):
            exp = np.zeros_like(q0, dtype=np.int64)
            for n in range(N):
                others = np.delete(q0, n, axis=1).astype(np.int64)
                s = np.prod(np.sign(others), axis=1)
                mag = np.minimum(np.abs(others).min(axis=1), qm)
                exp[:, n] = q0[:, n] + s * _rule_g(rule, mag, kw.get("offset", 0), kw.get("norm_num", 3),
                                                   kw.get("norm_shift", 2))
            for form in FORMS:
                r = orc.decode_int(code, q0, form=form, rule=rule, msg_sat=qm, max_iter=1, early_stop=0, **kw)
                if not np.array_equal(r.z.astype(np.int64), exp):
                    bad.append((form, rule, N, qm))
    return bad


def test_hamming_saturated_traces(oracle_lib):
    assert hamming_failures(oracle) == []


def test_single_check_saturated_closed_form(oracle_lib):
    assert single_check_failures(oracle) == []


def test_saturation_changes_the_trace(oracle_lib):
    """The Qm = 2 trace differs from the unsaturated one (so it tests the clamp):
    row 1's B after one iteration is 2, not 3."""
    assert GOLD["plain_qm2"]["state1_B"] != GOLD["plain"]["state1_B"]
    assert GOLD["plain_qm2"]["Z1"] != GOLD["plain"]["Z1"]
    assert GOLD["offset1_qm2"]["Z1"] != GOLD["offset1"]["Z1"]


# ------------------------------------------------------------------- mutants

_SAT = "return (p->msg_sat > 0 && mag > p->msg_sat) ? p->msg_sat : mag;"
_MUTANTS = {
    "clamp to Qm - 1": [(_SAT, "return (p->msg_sat > 0 && mag > p->msg_sat - 1) ? p->msg_sat - 1 : mag;")],
    "clamp to Qm + 1": [(_SAT, "return (p->msg_sat > 0 && mag > p->msg_sat + 1) ? p->msg_sat + 1 : mag;")],
    "no clamp": [(_SAT, "return mag;")],
    # the clamp moved behind the normalized / offset rule
    "clamp after the rule": [
        (_SAT, "return mag;"),
        ("static int64_t modify_i(const orc_iparams *p, int64_t mag) {",
         "static int64_t modify_i0(const orc_iparams *p, int64_t mag);\n"
         "static int64_t modify_i(const orc_iparams *p, int64_t mag) {\n"
         "  int64_t r = modify_i0(p, mag);\n"
         "  return (p->msg_sat > 0 && r > p->msg_sat) ? p->msg_sat : r;\n}\n"
         "static int64_t modify_i0(const orc_iparams *p, int64_t mag) {"),
    ],
}


def _load_mutant(path):
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.orc_decode_int.argtypes = [P, P, ctypes.c_int32, P, ctypes.c_int32, P, P, P, P, P, P, ctypes.c_int32]
    lib.orc_decode_int.restype = ctypes.c_int
    return lib


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_pins_reject_saturation_mutants(oracle_lib, tmp_path, monkeypatch, name):
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
    monkeypatch.setattr(oracle, "_lib", _load_mutant(so))
    failures = hamming_failures(oracle) + single_check_failures(oracle)
    assert failures, f"the saturation pins accept the mutant '{name}'"
