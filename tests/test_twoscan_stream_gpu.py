"""The two-scan algorithm of Section III (Eq. (1) horizontal scan, Eq. (2)
vertical scan) with the frame state in device memory, for codes of any size: its
check messages stored per edge (LDPC_FORM_TWO_SCAN, kernel STREAM) or in the
Section V form (LDPC_FORM_TWO_SCAN_1BIT).  Both must equal the literal two-scan
oracle bit for bit: decisions, iteration counts, flags and posteriors."""
import numpy as np
import pytest

from paper_cs_0609090_gb300 import inputs as I
from gpu_helpers import assert_int_parity, gpu_decode, oracle_int

pytestmark = pytest.mark.gpu

TWO_SCAN_FORMS = (("two_scan", "stream"), ("two_scan_1bit", "auto"))


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_cs_0609090_gb300 import ldpc
    return ldpc


def _run(L, w, q0, form, kernel, p):
    h = L.Code.from_inputs(w.code)
    g = gpu_decode(h, w.code.n_vars, q0, L.make_params(form=form, kernel=kernel, **p))
    assert_int_parity(g, oracle_int(w.code, q0, "two_scan", p))
    return g


@pytest.mark.parametrize("form,kernel", TWO_SCAN_FORMS)
@pytest.mark.parametrize("early_stop", [1, 0])
def test_small_codes(L, form, kernel, early_stop):
    """(3,6) N=1008 (check degree 6) and the QC N=7493 code (check degrees 14,
    15: the 16-byte Section V state), ragged frame counts."""
    w = I.make_workload("reg36_n1008", n_frames=301, ebn0_db=1.8)
    _run(L, w, w.q0, form, kernel, dict(w.params, early_stop=early_stop))
    w = I.make_workload("qc_n7493", n_frames=67, ebn0_db=2.0)
    _run(L, w, w.q0, form, kernel, dict(w.params, early_stop=early_stop))


@pytest.mark.parametrize("form,kernel", TWO_SCAN_FORMS)
def test_edge_cases(L, form, kernel):
    w = I.make_workload("reg36_n1008", n_frames=65, ebn0_db=1.0)
    for F in (1, 2, 65):
        _run(L, w, w.q0[:F], form, kernel, w.params)
    _run(L, w, w.q0[:5], form, kernel, dict(w.params, max_iter=0))
    _run(L, w, w.q0[:5], form, kernel, dict(w.params, max_iter=1, early_stop=0))
    g = _run(L, w, I.noiseless(w.codewords, 31), form, kernel, w.params)
    assert np.all(g["iters"] == 0)


@pytest.mark.parametrize("form,kernel", TWO_SCAN_FORMS)
def test_irregular_64800(L, form, kernel):
    """The N=64800 staircase code (check degrees 6, 7; variable degrees 1-8),
    with and without early stop."""
    w = I.make_workload("irr_n64800", n_frames=9, frame_seed=4)
    for es in (0, 1):
        _run(L, w, w.q0, form, kernel, dict(w.params, early_stop=es, max_iter=20))


@pytest.mark.parametrize("form,kernel", TWO_SCAN_FORMS)
def test_irr_64800_full_batch_sampled(L, form, kernel):
    """1024 frames, 50 iterations (the benchmarked comparator), sampled frames."""
    w = I.make_workload("irr_n64800")
    p = dict(w.params, early_stop=0)
    h = L.Code.from_inputs(w.code)
    g = gpu_decode(h, w.code.n_vars, w.q0, L.make_params(form=form, kernel=kernel, **p))
    frames = np.array([0, 1, 511, 1022, 1023])
    assert_int_parity({k: v[frames] for k, v in g.items()}, oracle_int(w.code, w.q0[frames], "two_scan", p))
