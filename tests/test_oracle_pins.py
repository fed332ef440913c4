"""Pins of the CPU oracle against facts fixed by the paper and by mathematics,
independent of the oracle's own code:

* hand-worked (7,4) Hamming decodes (tests/golden/hamming74_min_sum.json);
* noise-free frames stop before the first iteration;
* the equivalence of the two-scan, single-scan and Section V forms;
* exact max-marginals / ML decisions of min-sum on cycle-free codes
  (exhaustive enumeration of codewords);
* closed forms for a single parity check and a repetition code;
* scale, permutation and channel-symmetry invariants and the posterior bound.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import brute_force as bf
from paper_cs_0609090_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hamming74_min_sum.json")))
FORMS = ["two_scan", "ss_fixed", "ss_1bit"]


@pytest.fixture(scope="module")
def ham():
    return I.from_rows(GOLD["code"]["n_vars"], GOLD["code"]["rows"])


def _q0():
    return np.array([GOLD["q0"]], dtype=np.int32)


# ----------------------------------------------------------------- Hamming


@pytest.mark.parametrize("form", FORMS)
def test_hamming_plain_trace(oracle_lib, ham, form):
    g = GOLD["plain"]
    r0 = oracle.decode_int(ham, _q0(), form=form, rule="plain", max_iter=0, early_stop=0)
    assert r0.bits[0].tolist() == g["k0_bits"] and r0.ok[0] == g["k0_syndrome_ok"]
    assert r0.iters[0] == 0 and r0.z[0].tolist() == GOLD["q0"]
    r1 = oracle.decode_int(ham, _q0(), form=form, rule="plain", max_iter=1, early_stop=0,
                           want_l=True, want_state=(form == "ss_1bit"))
    assert r1.z[0].tolist() == g["Z1"]
    assert r1.bits[0].tolist() == g["k1_bits"]          # Z_1 = 0 decides bit 1
    assert r1.ok[0] == g["k1_syndrome_ok"] and r1.iters[0] == 1
    assert r1.l[0].tolist() == sum(g["L1"], [])
    if form == "ss_1bit":
        st = r1.state[0]
        assert st[:, 0].tolist() == g["state1_A"]
        assert st[:, 1].tolist() == g["state1_B"]
        assert st[:, 2].tolist() == g["state1_idx"]
        assert st[:, 3].tolist() == g["state1_signword"]
    r2 = oracle.decode_int(ham, _q0(), form=form, rule="plain", max_iter=2, early_stop=0, want_l=True)
    assert r2.z[0].tolist() == g["Z2"]
    assert r2.l[0].tolist() == sum(g["L2"], [])
    rf = oracle.decode_int(ham, _q0(), form=form, rule="plain", max_iter=20, early_stop=1)
    assert rf.bits[0].tolist() == g["final_bits"]
    assert rf.iters[0] == g["final_iters"] and rf.ok[0] == g["final_ok"]


@pytest.mark.parametrize("form", FORMS)
def test_hamming_offset_and_normalized(oracle_lib, ham, form):
    g = GOLD["offset1"]
    r = oracle.decode_int(ham, _q0(), form=form, rule="offset", offset=1, max_iter=1, early_stop=0,
                          want_l=True)
    assert r.z[0].tolist() == g["Z1"] and r.l[0].tolist() == sum(g["L1"], [])
    r = oracle.decode_int(ham, _q0(), form=form, rule="offset", offset=1, max_iter=10)
    assert (r.iters[0], r.ok[0]) == (g["final_iters"], g["final_ok"])
    g = GOLD["normalized_int_3_over_4"]
    r = oracle.decode_int(ham, _q0(), form=form, rule="normalized", norm_num=3, norm_shift=2,
                          max_iter=10)
    assert (r.iters[0], r.ok[0]) == (g["final_iters"], g["final_ok"])
    assert r.z[0].tolist() == g["Z1"]
    g = GOLD["normalized_float_0p75"]
    r = oracle.decode_f64(ham, _q0().astype(float), form=form, rule="normalized", lam=0.75,
                          max_iter=10)
    assert r.z[0].tolist() == g["Z1"]
    assert (r.iters[0], r.ok[0]) == (g["final_iters"], g["final_ok"])


def test_hamming_plain_f64_matches_int(oracle_lib, ham):
    g = GOLD["plain"]
    for form in FORMS:
        r = oracle.decode_f64(ham, _q0().astype(float), form=form, rule="plain", max_iter=2,
                              early_stop=0)
        assert r.z[0].tolist() == g["Z2"]


# ------------------------------------------------------ closed forms


def test_single_parity_check_closed_form(oracle_lib):
    """One check over all N variables: after one iteration
    Z_n = q0_n + prod_{n' != n} sgn(q0_n') * min_{n' != n} |q0_n'|."""
    rng = np.random.default_rng(5)
    N = 9
    code = I.from_rows(N, [list(range(N))])
    q0 = rng.integers(-40, 41, size=(200, N)).astype(np.int32)
    for form in FORMS:
        r = oracle.decode_int(code, q0, form=form, rule="plain", msg_sat=0, max_iter=1, early_stop=0)
        for f in range(0, 200, 7):
            for n in range(N):
                others = np.delete(q0[f], n)
                expect = q0[f, n] + np.prod(np.sign(others)) * np.abs(others).min()
                assert r.z[f, n] == expect


def test_repetition_code_sums_llrs(oracle_lib):
    """Repetition code (checks x_i = x_{i+1}): a chain, so after N-1 iterations
    every posterior equals the sum of all channel values."""
    N = 6
    code = I.from_rows(N, [[i, i + 1] for i in range(N - 1)])
    rng = np.random.default_rng(2)
    q0 = rng.integers(-30, 31, size=(100, N)).astype(np.int32)
    for form in FORMS:
        r = oracle.decode_int(code, q0, form=form, rule="plain", msg_sat=0, max_iter=N, early_stop=0)
        assert np.array_equal(r.z, np.repeat(q0.sum(axis=1, keepdims=True), N, axis=1))


# --------------------------------------------------------- noise-free frames


@pytest.mark.parametrize("wl", ["reg36_n1008", "qc_n7493", "irr_n64800"])
def test_noise_free_frames_stop_at_zero(oracle_lib, wl):
    w = I.make_workload(wl, n_frames=3, with_llr=True)
    q0 = I.noiseless(w.codewords, w.qc).astype(np.int32)
    for form in FORMS:
        r = oracle.decode_int(w.code, q0, form=form, rule=w.params["rule"],
                              offset=w.params.get("offset", 0), msg_sat=w.params["msg_sat"],
                              max_iter=w.params["max_iter"], early_stop=1)
        assert np.all(r.iters == 0) and np.all(r.ok == 1)
        assert np.array_equal(r.z, q0) and np.array_equal(r.bits, w.codewords)


# ------------------------------------------------------------- equivalence


def _int_kwargs(w):
    p = w.params
    return dict(rule=p["rule"], offset=p.get("offset", 0), norm_num=p.get("norm_num", 3),
                norm_shift=p.get("norm_shift", 2), msg_sat=p["msg_sat"], max_iter=p["max_iter"])


@pytest.mark.parametrize("wl,F", [("reg36_n1008", 1000), ("qc_n7493", 48)])
@pytest.mark.parametrize("early_stop", [0, 1])
def test_three_forms_agree(oracle_lib, wl, F, early_stop):
    """Section IV / V: the single scan and its Section V form are equivalent to
    the two-scan min-sum (exact in integers with an unsaturated posterior)."""
    w = I.make_workload(wl, n_frames=F, ebn0_db=I.WORKLOADS[wl][3] - 0.5)
    kw = _int_kwargs(w)
    res = [oracle.decode_int(w.code, w.q0, form=f, early_stop=early_stop, want_l=True, **kw)
           for f in FORMS]
    for r in res[1:]:
        for key in ("bits", "iters", "ok", "z", "l"):
            assert np.array_equal(res[0][key], r[key]), key
    assert res[0].ok.mean() < 1.0 or early_stop == 0  # some frames are hard


def test_three_forms_agree_irregular_staircase(oracle_lib):
    w = I.make_workload("irr_n64800", n_frames=2)
    kw = _int_kwargs(w)
    kw["max_iter"] = 6
    res = [oracle.decode_int(w.code, w.q0, form=f, early_stop=0, **kw) for f in FORMS]
    for r in res[1:]:
        assert np.array_equal(res[0].z, r.z) and np.array_equal(res[0].bits, r.bits)


def test_f64_forms_agree(oracle_lib):
    w = I.make_workload("reg36_n1008", n_frames=64, ebn0_db=1.5)
    res = [oracle.decode_f64(w.code, w.llr, form=f, rule="normalized", lam=0.75, max_iter=20,
                             early_stop=0) for f in FORMS]
    for r in res[1:]:
        assert np.allclose(res[0].z, r.z, rtol=1e-12, atol=1e-9)
    res = [oracle.decode_f64(w.code, w.llr, form=f, rule="offset", offset=0.5, max_iter=20,
                             early_stop=1) for f in FORMS]
    for r in res[1:]:
        assert np.array_equal(res[0].iters, r.iters)


# ------------------------------------------------------ brute force, trees


@pytest.mark.parametrize("seed", range(12))
def test_tree_codes_reach_max_marginals(oracle_lib, seed):
    """Cycle-free Tanner graph, plain min-sum, enough iterations, no saturation:
    Z_n equals the exhaustive max-marginal and x is the ML codeword."""
    N = 8 + seed % 9
    code = I.tree_code(N, seed)
    rows = [list(r) for r in code.rows()]
    cw = bf.codewords(N, rows)
    rng = np.random.default_rng(100 + seed)
    q0 = rng.integers(-20, 21, size=(64, N)).astype(np.int32)
    mm = bf.max_marginals(cw, q0)
    ml, _, tie = bf.ml_decode(cw, q0)
    for form in FORMS:
        r = oracle.decode_int(code, q0, form=form, rule="plain", msg_sat=0, max_iter=2 * N,
                              early_stop=0)
        assert np.array_equal(r.z, mm.astype(np.int64)), form
        assert np.array_equal(r.bits[~tie], ml[~tie])
        rd = oracle.decode_f64(code, q0.astype(float) * 0.37, form=form, rule="plain",
                               max_iter=2 * N, early_stop=0)
        assert np.allclose(rd.z, mm * 0.37, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_cyclic_codes_vs_ml(oracle_lib, seed):
    """Codes with cycles: every syndrome-satisfying output is a codeword whose
    correlation does not exceed the ML correlation; min-sum's frame errors are
    at least ML's."""
    N, M = 16, 8
    rng = np.random.default_rng(seed)
    rows = []
    for m in range(M):
        rows.append(sorted(rng.choice(N, size=4, replace=False).tolist()))
    code = I.from_rows(N, rows)
    cw = bf.codewords(N, rows)
    F = 400
    tx = cw[rng.integers(cw.shape[0], size=F)]
    q0 = (np.where(tx == 0, 4, -4) + rng.integers(-6, 7, size=(F, N))).astype(np.int32)
    ml, best, tie = bf.ml_decode(cw, q0)
    r = oracle.decode_int(code, q0, form="ss_1bit", rule="plain", msg_sat=0, max_iter=30)
    okf = r.ok == 1
    sset = {tuple(c) for c in cw}
    for f in np.nonzero(okf)[0]:
        assert tuple(r.bits[f]) in sset
    corr = ((1 - 2 * r.bits.astype(float)) * q0).sum(axis=1)
    assert np.all(corr[okf] <= best[okf] + 1e-9)
    fer_ms = np.mean(np.any(r.bits != tx, axis=1))
    fer_ml = np.mean(np.any(ml != tx, axis=1))
    assert fer_ms >= fer_ml


# ----------------------------------------------------------------- invariants


def test_scale_invariance_plain(oracle_lib):
    """Plain min-sum commutes with positive scaling of the channel values
    (Section II: the estimate sigma^2 does not matter)."""
    w = I.make_workload("reg36_n1008", n_frames=50, ebn0_db=1.5)
    q = w.q0.astype(np.int32)
    for form in FORMS:
        a = oracle.decode_int(w.code, q, form=form, rule="plain", msg_sat=0, max_iter=15)
        b = oracle.decode_int(w.code, 3 * q, form=form, rule="plain", msg_sat=0, max_iter=15)
        assert np.array_equal(3 * a.z, b.z) and np.array_equal(a.iters, b.iters)
        assert np.array_equal(a.bits, b.bits)


def test_permutation_invariance(oracle_lib):
    w = I.make_workload("reg36_n1008", n_frames=80, ebn0_db=1.8)
    kw = _int_kwargs(w)
    base = oracle.decode_int(w.code, w.q0, form="ss_1bit", **kw)
    pc, _ = I.permuted(w.code, seed=3, rows=True, positions=True)
    r = oracle.decode_int(pc, w.q0, form="ss_1bit", **kw)
    for key in ("bits", "iters", "ok", "z"):
        assert np.array_equal(base[key], r[key])
    pc, perm = I.permuted(w.code, seed=4, rows=False, positions=False, cols=True)
    q = np.zeros_like(w.q0)
    q[:, perm] = w.q0
    r = oracle.decode_int(pc, q, form="two_scan", **kw)
    assert np.array_equal(r.z[:, perm], base.z) and np.array_equal(r.iters, base.iters)


def test_channel_symmetry(oracle_lib):
    """Flipping q0 on the support of a codeword c flips every message sign on
    that support: at a fixed iteration count Z' = Z (1 - 2c) exactly, so the
    decisions are XORed with c wherever Z != 0."""
    w = I.make_workload("reg36_n1008", n_frames=100, ebn0_db=1.6, zero_codeword=True)
    kw = _int_kwargs(w)
    c = I.Encoder(w.code).random_codewords(1, seed=9)[0]
    s = np.where(c == 1, -1, 1)[None, :]
    for form in FORMS:
        a = oracle.decode_int(w.code, w.q0, form=form, early_stop=0, **kw)
        b = oracle.decode_int(w.code, w.q0.astype(np.int32) * s, form=form, early_stop=0, **kw)
        assert np.array_equal(b.z, a.z * s)
        nz = a.z != 0
        assert np.array_equal(b.bits[nz], (a.bits ^ c[None, :])[nz])


def test_posterior_bound(oracle_lib):
    """|Z_n - q0_n| <= deg(n) * Qm after any iteration."""
    w = I.make_workload("qc_n7493", n_frames=8, ebn0_db=1.5)
    kw = _int_kwargs(w)
    dv = w.code.col_degrees()
    for it in (1, 3, 7):
        kw["max_iter"] = it
        r = oracle.decode_int(w.code, w.q0, form="ss_1bit", early_stop=0, **kw)
        assert np.all(np.abs(r.z - w.q0) <= dv[None, :] * kw["msg_sat"])
