"""GPU vs oracle parity of the layered schedule (the single scan of Eq. (3)
with column-disjoint layers updating the posteriors in place): decisions,
iteration counts, syndrome flags and final posteriors bit-identical to the
layered oracle run with the library's own layer partition."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_cs_0609090_gb300 import inputs as I
from gpu_helpers import FORMS_INT, assert_int_parity, gpu_decode

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_cs_0609090_gb300 import ldpc
    return ldpc


def _oracle(code, q0, lay, p):
    return oracle.decode_layered_int(code, q0.astype(np.int32), lay, rule=p.get("rule", "offset"),
                                     offset=p.get("offset", 0), norm_num=p.get("norm_num", 3),
                                     norm_shift=p.get("norm_shift", 2), msg_sat=p.get("msg_sat", 127),
                                     max_iter=p["max_iter"], early_stop=p.get("early_stop", 1))


def _run(L, code, q0, form, p, frames=None, layers=None):
    h = L.Code.from_inputs(code)
    if layers is not None:
        L.ldpc_code_set_layers(h.handle, layers)
    n, lay = L.ldpc_code_layers(h.handle, code.n_checks)
    assert n == lay.max() + 1
    g = gpu_decode(h, code.n_vars, q0, L.make_params(form=form, schedule="layered", **p))
    sel = slice(None) if frames is None else frames
    g = {k: v[sel] for k, v in g.items()}
    assert_int_parity(g, _oracle(code, q0[sel], lay, p))
    return g, lay


def test_hamming_layered_golden(L):
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hamming74_min_sum.json")))
    code = I.from_rows(7, gold["code"]["rows"])
    q0 = np.array([gold["q0"]] * 3, dtype=np.int8)
    h = L.Code.from_inputs(code)
    assert L.ldpc_code_layers(h.handle, 3)[1].tolist() == gold["layered_plain"]["layers"]
    for form in FORMS_INT:
        g = gpu_decode(h, 7, q0, L.make_params(form=form, rule="plain", max_iter=1, early_stop=0, schedule="layered"))
        assert g["z"][0].tolist() == gold["layered_plain"]["Z1"]
        g = gpu_decode(h, 7, q0, L.make_params(form=form, rule="plain", max_iter=2, early_stop=0, schedule="layered"))
        assert g["z"][0].tolist() == gold["layered_plain"]["Z2_no_early_stop"]
        g = gpu_decode(h, 7, q0, L.make_params(form=form, rule="plain", max_iter=20, schedule="layered"))
        assert g["iters"].tolist() == [1, 1, 1] and g["ok"].tolist() == [1, 1, 1]
        g = gpu_decode(h, 7, q0, L.make_params(form=form, rule="offset", offset=1, max_iter=1, early_stop=0,
                                               schedule="layered"))
        assert g["z"][0].tolist() == gold["layered_offset1"]["Z1"]


@pytest.mark.parametrize("form", FORMS_INT)
@pytest.mark.parametrize("early_stop", [1, 0])
def test_regular_1008_layered(L, form, early_stop):
    w = I.make_workload("reg36_n1008", n_frames=301, ebn0_db=1.8)
    _run(L, w.code, w.q0, form, dict(w.params, early_stop=early_stop))


@pytest.mark.parametrize("form", FORMS_INT)
def test_qc_7493_layered(L, form):
    w = I.make_workload("qc_n7493", n_frames=203, ebn0_db=3.0, frame_seed=4)
    _run(L, w.code, w.q0, form, w.params)
    _run(L, w.code, w.q0[:33], form, dict(w.params, early_stop=0, max_iter=12))


def test_qc_7493_block_row_layers(L):
    """The 24 block rows of the quasi-cyclic code as layers (set through the ABI)."""
    w = I.make_workload("qc_n7493", n_frames=64, ebn0_db=3.0)
    block_rows = (np.arange(w.code.n_checks) // 127).astype(np.int32)
    g, lay = _run(L, w.code, w.q0, "ss_1bit", w.params, layers=block_rows)
    assert lay.tolist() == block_rows.tolist()


@pytest.mark.parametrize("form", FORMS_INT)
def test_irr_64800_layered(L, form):
    w = I.make_workload("irr_n64800", n_frames=5, frame_seed=2)
    _run(L, w.code, w.q0, form, dict(w.params, max_iter=12))


@pytest.mark.parametrize("form", FORMS_INT)
def test_layered_edge_cases(L, form):
    w = I.make_workload("reg36_n1008", n_frames=19, ebn0_db=1.0)
    _run(L, w.code, w.q0[:1], form, w.params)                           # one frame
    _run(L, w.code, w.q0, form, dict(w.params, max_iter=0))
    g, _ = _run(L, w.code, I.noiseless(w.codewords, 31), form, w.params)
    assert np.all(g["iters"] == 0) and np.all(g["ok"] == 1)
    rng = np.random.default_rng(8)
    q = rng.integers(-128, 128, size=(17, w.code.n_vars)).astype(np.int8)
    _run(L, w.code, q, form, dict(w.params, msg_sat=127, rule="plain", early_stop=0, max_iter=9))
    _run(L, w.code, w.q0, form, dict(w.params, rule="normalized", norm_num=5, norm_shift=3))


def test_layered_rejections(L):
    import torch
    w = I.make_workload("reg36_n1008", n_frames=2)
    h = L.Code.from_inputs(w.code)
    q = torch.from_numpy(w.q0).cuda()
    for kw in (dict(form="two_scan"), dict(dtype="f32"), dict(kernel="stream")):
        with pytest.raises(L.LdpcError) as e:
            L.decode(h, q if kw.get("dtype") != "f32" else q.float(),
                     L.make_params(schedule="layered", **dict(w.params, **kw)))
        assert e.value.status == L.LDPC_ERR_UNSUPPORTED
    bad = np.zeros(w.code.n_checks, np.int32)      # every check in one layer: they share variables
    with pytest.raises(L.LdpcError) as e:
        L.ldpc_code_set_layers(h.handle, bad)
    assert e.value.status == L.LDPC_ERR_INVALID_ARG
    n, lay = L.ldpc_code_layers(h.handle, w.code.n_checks)      # the old partition stays
    assert n == lay.max() + 1 > 1


def test_layered_converges_in_fewer_iterations(L):
    """Same frames, same code: mean iterations to a codeword, layered against flooding."""
    w = I.make_workload("qc_n7493", n_frames=512, ebn0_db=3.0, frame_seed=9)
    h = L.Code.from_inputs(w.code)
    a = gpu_decode(h, w.code.n_vars, w.q0, L.make_params(schedule="layered", **w.params), want_llr=False)
    b = gpu_decode(h, w.code.n_vars, w.q0, L.make_params(**w.params), want_llr=False)
    assert a["iters"].mean() < 0.75 * b["iters"].mean()
    assert a["ok"].sum() >= 0.98 * b["ok"].sum()   # (497 against 501 frames on one run)
