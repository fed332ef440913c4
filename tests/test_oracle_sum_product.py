"""Pins of the oracle's sum-product check rule (the log-domain rule that
min-sum approximates; the accuracy reference of the min-sum decoders), against what does not
depend on it:
* cycle-free codes: the posteriors equal the exact a-posteriori LLRs (brute
  force over all codewords) after enough iterations;
* one check, one iteration: L_j = 2 atanh(prod over the other positions of
  tanh(q/2)) (the tanh form, not the phi form the oracle uses);
* |L_sum-product| <= |L_min-sum| for the same inputs, with equal signs;
* the two-scan and single-scan schedules give the same posteriors."""
import numpy as np
import pytest

import oracle
from oracle import brute_force as bf
from paper_cs_0609090_gb300 import inputs as I


@pytest.mark.parametrize("seed", range(10))
def test_tree_codes_reach_app_llr(seed):
    N = 8 + seed % 9
    code = I.tree_code(N, seed)
    rows = [list(r) for r in code.rows()]
    cw = bf.codewords(N, rows)
    q0 = np.random.default_rng(300 + seed).uniform(-1.5, 1.5, size=(32, N))   # |Z| < 30: no saturation
    app = bf.app_llr(cw, q0)
    for form in ("two_scan", "ss_fixed"):
        r = oracle.decode_f64(code, q0, form=form, rule="sum_product", max_iter=2 * N, early_stop=0)
        assert np.allclose(r.z, app, rtol=1e-9, atol=1e-9), (form, np.abs(r.z - app).max())


def test_single_check_tanh_closed_form():
    code = I.from_rows(6, [[0, 1, 2, 3, 4, 5]])
    q0 = np.random.default_rng(7).normal(0.5, 2.0, size=(40, 6))
    r = oracle.decode_f64(code, q0, form="ss_fixed", rule="sum_product", max_iter=1, early_stop=0, want_l=True)
    for f in range(q0.shape[0]):
        t = np.tanh(np.clip(q0[f], -oracle.SPA_SAT, oracle.SPA_SAT) / 2)
        want = np.array([2 * np.arctanh(np.prod(np.delete(t, j))) for j in range(6)])
        assert np.allclose(r.l[f], want, rtol=1e-10, atol=1e-12)
        assert np.allclose(r.z[f], q0[f] + want, rtol=1e-10, atol=1e-12)


def test_magnitudes_below_min_sum():
    w = I.make_workload("reg36_n1008", n_frames=16, ebn0_db=1.5)
    a = oracle.decode_f64(w.code, w.llr, form="ss_fixed", rule="sum_product", max_iter=1, early_stop=0,
                          want_l=True)
    b = oracle.decode_f64(w.code, w.llr, form="ss_fixed", rule="plain", max_iter=1, early_stop=0, want_l=True)
    assert np.all(np.abs(a.l) <= np.abs(b.l) + 1e-12)
    nz = np.abs(a.l) > 1e-12
    assert np.array_equal(np.sign(a.l[nz]), np.sign(b.l[nz]))


def test_schedules_agree_and_one_bit_form_is_rejected():
    w = I.make_workload("reg36_n1008", n_frames=12, ebn0_db=1.5)
    a = oracle.decode_f64(w.code, w.llr, form="two_scan", rule="sum_product", max_iter=15, early_stop=0)
    b = oracle.decode_f64(w.code, w.llr, form="ss_fixed", rule="sum_product", max_iter=15, early_stop=0)
    assert np.allclose(a.z, b.z, rtol=1e-9, atol=1e-9)
    with pytest.raises(ValueError):
        oracle.decode_f64(w.code, w.llr, form="ss_1bit", rule="sum_product", max_iter=3)
