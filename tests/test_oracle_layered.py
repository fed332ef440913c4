"""Pins of the layered-schedule oracle (the single scan of Eq. (3) with checks
grouped into layers of column-disjoint checks that update the posteriors in
place), against what does not depend on it:
* hand-worked (7,4) Hamming iterations (tests/golden/hamming74_min_sum.json);
* one layer of pairwise disjoint checks is the flooding schedule (pinned in
  test_oracle_pins.py);
* on cycle-free codes min-sum reaches the exhaustive max-marginals under any
  schedule;
* the order of the checks inside a layer does not matter, the order of the
  layers does;
* the layer partition is validated (checks of a layer must share no variable)."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import brute_force as bf
from paper_cs_0609090_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hamming74_min_sum.json")))


def greedy_layers(code):
    """Checks in row order, each into the lowest layer none of whose checks
    shares a variable with it."""
    used = []   # per layer: set of variables
    layer = np.zeros(code.n_checks, np.int32)
    for m, row in enumerate(code.rows()):
        vs = set(int(v) for v in row)
        for ell, u in enumerate(used):
            if not (u & vs):
                u |= vs
                layer[m] = ell
                break
        else:
            used.append(set(vs))
            layer[m] = len(used) - 1
    return layer


def test_hamming_layered_hand_worked():
    code = I.from_rows(7, GOLD["code"]["rows"])
    q0 = np.array([GOLD["q0"]], np.int32)
    g = GOLD["layered_plain"]
    lay = np.array(g["layers"], np.int32)
    assert np.array_equal(greedy_layers(code), lay)
    r = oracle.decode_layered_int(code, q0, lay, rule="plain", max_iter=1, early_stop=0, want_l=True)
    assert r.z[0].tolist() == g["Z1"]
    assert r.l[0].tolist() == [v for row in g["L1"] for v in row]
    assert r.ok[0] == g["k1_syndrome_ok"]
    r = oracle.decode_layered_int(code, q0, lay, rule="plain", max_iter=20, early_stop=1)
    assert r.iters[0] == g["final_iters"] and r.bits[0].tolist() == [0] * 7
    r = oracle.decode_layered_int(code, q0, lay, rule="plain", max_iter=2, early_stop=0)
    assert r.z[0].tolist() == g["Z2_no_early_stop"]
    r = oracle.decode_layered_int(code, q0, lay, rule="offset", offset=1, max_iter=1, early_stop=0)
    assert r.z[0].tolist() == GOLD["layered_offset1"]["Z1"]


@pytest.mark.parametrize("rule", ["plain", "offset", "normalized"])
def test_single_layer_is_flooding(rule):
    """Pairwise disjoint checks in one layer: the in-place updates of different
    checks never meet, so the layered decode equals the flooding single scan."""
    rng = np.random.default_rng(4)
    N = 72
    perm = rng.permutation(N)
    rows = [perm[6 * i:6 * i + 6].tolist() for i in range(12)]
    code = I.from_rows(N, rows, sort=False)
    q0 = rng.integers(-12, 13, size=(40, N)).astype(np.int32)
    kw = dict(rule=rule, offset=1, norm_num=3, norm_shift=2, msg_sat=9, max_iter=7)
    for es in (0, 1):
        a = oracle.decode_layered_int(code, q0, np.zeros(12, np.int32), early_stop=es, want_l=True, **kw)
        b = oracle.decode_int(code, q0, form="ss_fixed", early_stop=es, want_l=True, **kw)
        for key in ("bits", "iters", "ok", "z", "l"):
            assert np.array_equal(a[key], b[key]), key


@pytest.mark.parametrize("seed", range(8))
def test_tree_codes_reach_max_marginals_layered(seed):
    N = 8 + seed % 9
    code = I.tree_code(N, seed)
    rows = [list(r) for r in code.rows()]
    cw = bf.codewords(N, rows)
    q0 = np.random.default_rng(200 + seed).integers(-20, 21, size=(48, N)).astype(np.int32)
    mm = bf.max_marginals(cw, q0)
    r = oracle.decode_layered_int(code, q0, greedy_layers(code), rule="plain", msg_sat=0, max_iter=2 * N,
                                  early_stop=0)
    assert np.array_equal(r.z, mm.astype(np.int64))


def test_order_inside_layers_is_free_order_of_layers_is_not():
    w = I.make_workload("reg36_n1008", n_frames=24, ebn0_db=1.5)
    code, q0 = w.code, w.q0
    lay = greedy_layers(code)
    kw = dict(rule="offset", offset=1, msg_sat=31, max_iter=6, early_stop=0)
    base = oracle.decode_layered_int(code, q0, lay, want_l=True, **kw)
    # permute the checks (each keeps its layer) and the positions inside each check
    rng = np.random.default_rng(1)
    order = rng.permutation(code.n_checks)
    rows = [list(code.rows())[m] for m in order]
    pc = I.from_rows(code.n_vars, rows, sort=False)
    r = oracle.decode_layered_int(pc, q0, lay[order], want_l=True, **kw)
    for key in ("bits", "iters", "ok", "z"):
        assert np.array_equal(r[key], base[key]), key
    rp = np.asarray(pc.row_ptr)
    lb = base.l.reshape(q0.shape[0], -1)
    rpb = np.asarray(code.row_ptr)
    for i, m in enumerate(order[:50]):
        assert np.array_equal(r.l[:, rp[i]:rp[i + 1]], lb[:, rpb[m]:rpb[m + 1]])
    # reversed layer order: a different schedule, different posteriors
    rev = lay.max() - lay
    r2 = oracle.decode_layered_int(code, q0, rev, **kw)
    assert not np.array_equal(r2.z, base.z)


def test_layers_must_be_column_disjoint():
    code = I.from_rows(7, GOLD["code"]["rows"])
    with pytest.raises(ValueError):
        oracle.decode_layered_int(code, np.zeros((1, 7), np.int32), np.array([0, 0, 1], np.int32))


def test_layered_needs_fewer_iterations():
    """The layered schedule's known property (cited in Section I): on the QC code
    at 3.0 dB it reaches a codeword in fewer iterations on average than flooding
    (measured: 4.9 against 8.7 on these frames)."""
    w = I.make_workload("qc_n7493", n_frames=48, ebn0_db=3.0)
    p = w.params
    kw = dict(rule=p["rule"], offset=p["offset"], msg_sat=p["msg_sat"], max_iter=30, early_stop=1)
    a = oracle.decode_layered_int(w.code, w.q0, greedy_layers(w.code), **kw)
    b = oracle.decode_int(w.code, w.q0, form="ss_fixed", **kw)
    assert a.iters.mean() < 0.8 * b.iters.mean()
    assert a.ok.sum() >= b.ok.sum() - 1
