"""GPU vs oracle parity of the int8 single-scan decoders (fixed-point form of
Section IV and 1-bit form of Section V): decisions, iteration counts, syndrome
flags and final posteriors must be bit-identical."""
import numpy as np
import pytest

from paper_cs_0609090_gb300 import inputs as I
from gpu_helpers import FORMS_INT, KERNELS_INT, assert_int_parity, gpu_decode, oracle_int

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_cs_0609090_gb300 import ldpc
    return ldpc


def _run(L, code, q0, form, p, frames=None, kernels=("auto",)):
    h = L.Code.from_inputs(code)
    o = oracle_int(code, q0 if frames is None else q0[frames], form, p)
    for kern in kernels:
        params = L.make_params(form=form, kernel=kern, **p)
        g = gpu_decode(h, code.n_vars, q0, params)
        if frames is not None:
            g = {k: v[frames] for k, v in g.items()}
        assert_int_parity(g, o)
    return g


@pytest.mark.parametrize("form", FORMS_INT)
def test_hamming_golden(L, form):
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hamming74_min_sum.json")))
    code = I.from_rows(7, gold["code"]["rows"])
    q0 = np.array([gold["q0"]] * 3, dtype=np.int8)
    h = L.Code.from_inputs(code)
    for it, key in ((1, "Z1"), (2, "Z2")):
        g = gpu_decode(h, 7, q0, L.make_params(form=form, rule="plain", max_iter=it, early_stop=0))
        assert g["z"][0].tolist() == gold["plain"][key]
    g = gpu_decode(h, 7, q0, L.make_params(form=form, rule="plain", max_iter=20, early_stop=1))
    assert g["iters"].tolist() == [2, 2, 2] and g["ok"].tolist() == [1, 1, 1]
    g = gpu_decode(h, 7, q0, L.make_params(form=form, rule="offset", offset=1, max_iter=20))
    assert g["z"][0].tolist() == gold["offset1"]["Z1"] and g["iters"][0] == 1


@pytest.mark.parametrize("form", FORMS_INT)
@pytest.mark.parametrize("early_stop", [1, 0])
def test_regular_1008_full_batch(L, form, early_stop):
    w = I.make_workload("reg36_n1008")
    p = dict(w.params, early_stop=early_stop)
    _run(L, w.code, w.q0, form, p, kernels=KERNELS_INT)


@pytest.mark.parametrize("form", FORMS_INT)
@pytest.mark.parametrize("ebn0", [2.0, 2.5, 3.0])
def test_qc_7493(L, form, ebn0):
    w = I.make_workload("qc_n7493", n_frames=203, ebn0_db=ebn0, frame_seed=int(ebn0 * 10))
    _run(L, w.code, w.q0, form, w.params, kernels=KERNELS_INT)


@pytest.mark.parametrize("form", FORMS_INT)
def test_qc_7493_full_batch_sampled(L, form):
    """The full 4096-frame batch in the bench's launch configuration; the oracle
    checks a sample of frames spread over all CTAs and the ragged tail."""
    w = I.make_workload("qc_n7493")
    p = dict(w.params, early_stop=0)
    rng = np.random.default_rng(0)
    frames = np.unique(np.concatenate([rng.choice(w.n_frames, 40, replace=False),
                                       [0, 1, w.n_frames - 2, w.n_frames - 1]]))
    _run(L, w.code, w.q0, form, p, frames=frames, kernels=KERNELS_INT)


@pytest.mark.parametrize("form", FORMS_INT)
def test_edge_cases(L, form):
    w = I.make_workload("reg36_n1008", n_frames=7, ebn0_db=1.0)
    K = KERNELS_INT
    # one frame, odd frame count (ragged frame pair), max_iter = 0
    _run(L, w.code, w.q0[:1], form, w.params, kernels=K)
    _run(L, w.code, w.q0, form, w.params, kernels=K)
    _run(L, w.code, w.q0, form, dict(w.params, max_iter=0), kernels=K)
    _run(L, w.code, w.q0, form, dict(w.params, max_iter=1, early_stop=0), kernels=K)
    # noise-free frames stop before the first iteration
    q = I.noiseless(w.codewords, 31)
    g = _run(L, w.code, q, form, w.params, kernels=K)
    assert np.all(g["iters"] == 0) and np.all(g["ok"] == 1)
    # extreme channel values, full int8 range
    rng = np.random.default_rng(3)
    q = rng.integers(-128, 128, size=(9, w.code.n_vars)).astype(np.int8)
    _run(L, w.code, q, form, dict(w.params, msg_sat=127, rule="plain", early_stop=0, max_iter=12), kernels=K)


@pytest.mark.parametrize("form", FORMS_INT)
@pytest.mark.parametrize("rule", ["plain", "offset", "normalized"])
def test_rules_and_irregular_degrees(L, form, rule):
    """Rows of degree 2..32, variables of degree 0 and 1, all three rules."""
    rng = np.random.default_rng(11)
    N = 600
    rows = []
    for m in range(120):
        d = [2, 3, 7, 16, 31, 32][m % 6]
        rows.append(rng.choice(N - 5, size=d, replace=False))   # last 5 variables unused
    rows.append([N - 5, 0])                                       # variable N-5 has degree 1
    code = I.from_rows(N, rows, sort=False)
    q0 = rng.integers(-20, 25, size=(37, N)).astype(np.int8)
    p = dict(rule=rule, offset=2, norm_num=3, norm_shift=2, msg_sat=63, max_iter=9, early_stop=1)
    _run(L, code, q0, form, p)
    _run(L, code, q0, form, dict(p, early_stop=0))
    # the same rules on a code the packed kernel accepts (row degree <= 16)
    rows16 = [r[:16] for r in rows]
    code16 = I.from_rows(N, rows16, sort=False)
    _run(L, code16, q0, form, p, kernels=KERNELS_INT)
    _run(L, code16, q0, form, dict(p, early_stop=0, rule=rule, norm_num=5, norm_shift=3), kernels=KERNELS_INT)


@pytest.mark.parametrize("seed", range(3))
def test_tree_and_permuted_codes(L, seed):
    code = I.tree_code(18, seed)
    rng = np.random.default_rng(seed)
    q0 = rng.integers(-20, 21, size=(33, 18)).astype(np.int8)
    for form in FORMS_INT:
        _run(L, code, q0, form, dict(rule="plain", msg_sat=127, max_iter=36, early_stop=0), kernels=KERNELS_INT)
    w = I.make_workload("reg36_n1008", n_frames=64, ebn0_db=1.7)
    pc, _ = I.permuted(w.code, seed=seed)
    for form in FORMS_INT:
        _run(L, pc, w.q0, form, w.params, kernels=KERNELS_INT)


def test_forced_kernel_rejects_ineligible_code(L):
    """The packed kernel refuses codes whose magnitudes could reach 2048."""
    rng = np.random.default_rng(1)
    rows = [rng.choice(200, size=20, replace=False) for _ in range(40)]   # degree 20 > 16
    code = I.from_rows(200, rows, sort=False)
    h = L.Code.from_inputs(code)
    import torch
    q = torch.zeros((2, 200), dtype=torch.int8, device="cuda")
    with pytest.raises(L.LdpcError) as e:
        L.decode(h, q, L.make_params(kernel="onchip_half", max_iter=3))
    assert e.value.status == L.LDPC_ERR_UNSUPPORTED


def test_frame_resident_kernels_reject_large_code(L):
    """A code whose frame state exceeds one SM cannot be forced onto an on-chip kernel."""
    w = I.make_workload("irr_n64800", n_frames=1, with_llr=False)
    h = L.Code.from_inputs(w.code)
    import torch
    q = torch.zeros((2, w.code.n_vars), dtype=torch.int8, device="cuda")
    for kern in ("onchip_half", "onchip_int"):
        with pytest.raises(L.LdpcError) as e:
            L.decode(h, q, L.make_params(kernel=kern, **w.params))
        assert e.value.status == L.LDPC_ERR_UNSUPPORTED


@pytest.mark.parametrize("early_stop", [1, 0])
def test_two_scan_comparator(L, early_stop):
    """The GPU two-scan comparator (Eqs. (1)-(2)) against the oracle's literal two-scan."""
    for wl, F, eb in (("reg36_n1008", 300, 1.8), ("qc_n7493", 45, 2.0)):
        w = I.make_workload(wl, n_frames=F, ebn0_db=eb)
        _run(L, w.code, w.q0, "two_scan", dict(w.params, early_stop=early_stop))
    w = I.make_workload("reg36_n1008", n_frames=5, ebn0_db=1.0)
    _run(L, w.code, w.q0[:1], "two_scan", dict(w.params, early_stop=early_stop))
    _run(L, w.code, w.q0, "two_scan", dict(w.params, max_iter=0, early_stop=early_stop))


def test_two_scan_hamming_and_tree(L):
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hamming74_min_sum.json")))
    code = I.from_rows(7, gold["code"]["rows"])
    h = L.Code.from_inputs(code)
    q0 = np.array([gold["q0"]] * 3, dtype=np.int8)
    g = gpu_decode(h, 7, q0, L.make_params(form="two_scan", rule="plain", max_iter=2, early_stop=0))
    assert g["z"][0].tolist() == gold["plain"]["Z2"]
    tc = I.tree_code(16, 4)
    rng = np.random.default_rng(4)
    q = rng.integers(-20, 21, size=(17, 16)).astype(np.int8)
    _run(L, tc, q, "two_scan", dict(rule="plain", msg_sat=127, max_iter=32, early_stop=0))
    _run(L, tc, q, "two_scan", dict(rule="normalized", norm_num=3, norm_shift=2, msg_sat=100, max_iter=9))
