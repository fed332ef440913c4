"""Pins of the oracle pieces behind the learned offset decoder:
* Philox4x32-10 known-answer vectors (Random123 distribution of Salmon et al.);
* AWGN moments of the generated LLRs;
* the FP64 reverse-mode gradient against central finite differences of the
  oracle's (separately pinned) forward decode, against a closed form for one
  check, and its loss against the BCE of the forward's posterior."""
import numpy as np
import pytest

import oracle
from oracle import philox
from paper_cs_0609090_gb300 import inputs as I


def test_philox_known_answers():
    kat = [((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
           ((0xffffffff,) * 4, (0xffffffff, 0xffffffff), (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
           ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
            (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1))]
    for ctr, key, want in kat:
        got = philox.philox4x32_10(np.array([ctr], dtype=np.uint32), key)[0]
        assert tuple(int(x) for x in got) == want


def test_awgn_moments():
    """All-zero codeword: LLR = 2/s2 + 2 xi/sigma, so mean 2/s2 and variance 4/s2."""
    N, F, rate = 20000, 4, 0.5
    llr, eb = philox.awgn_llr(N, seed=7, first_frame=0, n_frames=F, lo=1.0, hi=3.0, rate=rate)
    assert np.all((eb >= 1.0) & (eb <= 3.0))
    for f in range(F):
        s2 = 1.0 / (2 * rate * 10 ** (eb[f] / 10))
        assert abs(llr[f].mean() - 2 / s2) < 4 * np.sqrt(4 / s2 / N)
        assert abs(llr[f].var() / (4 / s2) - 1) < 0.05


def _bce_sum(z):
    return float(np.sum(np.logaddexp(0.0, -z)))  # softplus(-Z), all-zero codeword


def _class_tab(code, beta_kc):
    deg = code.row_degrees()
    classes = sorted(set(deg.tolist()))
    cls = np.array([classes.index(d) for d in deg])
    return beta_kc[:, cls], cls, len(classes)


def test_learned_gradient_finite_differences():
    w = I.make_workload("qc_n7493", n_frames=12, ebn0_db=2.0, zero_codeword=True)
    K = 6
    rng = np.random.default_rng(3)
    beta_kc = rng.uniform(0.1, 0.6, size=(K, 2))
    tab, cls, C = _class_tab(w.code, beta_kc)
    loss, db, gap = oracle.learned_grad(w.code, w.llr, tab)
    z = oracle.decode_f64(w.code, w.llr, form="ss_fixed", rule="offset", beta_tab=tab, max_iter=K,
                          early_stop=0).z
    assert abs(loss - _bce_sum(z)) <= 1e-9 * abs(loss)
    # u moves by up to |du/dbeta| eps (large after a few iterations), so the step
    # is kept 1000x below the distance to the nearest kink
    eps = 1e-8
    keep = gap > 1000 * eps
    assert keep.sum() >= 3
    q = w.llr[keep]
    _, db, _ = oracle.learned_grad(w.code, q, tab)
    for k in range(K):
        for c in range(C):
            bp, bm = beta_kc.copy(), beta_kc.copy()
            bp[k, c] += eps
            bm[k, c] -= eps
            lp = _bce_sum(oracle.decode_f64(w.code, q, form="ss_1bit", rule="offset", beta_tab=_class_tab(
                w.code, bp)[0], max_iter=K, early_stop=0).z)
            lm = _bce_sum(oracle.decode_f64(w.code, q, form="ss_1bit", rule="offset", beta_tab=_class_tab(
                w.code, bm)[0], max_iter=K, early_stop=0).z)
            fd = (lp - lm) / (2 * eps)
            an = db[k, cls == c].sum()
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (k, c, fd, an)


def test_learned_gradient_single_check_closed_form():
    """One check over 5 variables, one iteration: Z_n = q_n + s_n relu(m_n - beta)
    with m_n the smallest |q| of the others; dLoss/dbeta = sum_n (1 - sigma(Z_n)) s_n [m_n > beta]."""
    code = I.from_rows(5, [[0, 1, 2, 3, 4]])
    rng = np.random.default_rng(1)
    q = rng.normal(1.0, 2.0, size=(7, 5))
    beta = 0.4
    loss, db, _ = oracle.learned_grad(code, q, np.array([[beta]]))
    want = 0.0
    for f in range(q.shape[0]):
        for n in range(5):
            o = np.delete(q[f], n)
            s, mn = np.prod(np.sign(o)), np.abs(o).min()
            zn = q[f, n] + s * max(mn - beta, 0.0)
            if mn > beta:
                want += (1 - 1 / (1 + np.exp(-zn))) * s
    assert abs(db[0, 0] - want) <= 1e-12 * max(1.0, abs(want))
