"""The persistent streaming decoder (LDPC_KERNEL_PERSISTENT): bit-exact parity
with the oracle on many groups of chunks, on frames that stop at different
iterations, and on the full N=7493 batch; and its failure path: the bounded wait
between work items gives up on a counter that nothing increments, reports
LDPC_ERR_TIMEOUT, and leaves the context usable for the next decode."""
import numpy as np
import pytest

from paper_cs_0609090_gb300 import inputs as I
from gpu_helpers import FORMS_INT, assert_int_parity, gpu_decode, oracle_int

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_cs_0609090_gb300 import ldpc
    return ldpc


@pytest.mark.parametrize("form", FORMS_INT)
def test_many_groups_mixed_stops(L, form):
    """1000 frames of the N=1008 code at a low Eb/N0 with early stop: 16 chunks in
    8 groups; frames stop anywhere from 0 to 20 iterations."""
    w = I.make_workload("reg36_n1008", n_frames=1000, ebn0_db=1.6, frame_seed=11)
    q = w.q0.copy()
    q[::7] = I.noiseless(w.codewords[::7], 31)  # some frames stop before the first iteration
    h = L.Code.from_inputs(w.code)
    g = gpu_decode(h, w.code.n_vars, q, L.make_params(form=form, kernel="persistent", **w.params))
    o = oracle_int(w.code, q, form, w.params)
    assert_int_parity(g, o)
    assert len(np.unique(o.iters)) > 5 and np.any(o.iters == 0) and np.any(o.ok == 0)


@pytest.mark.parametrize("form", FORMS_INT)
def test_qc_7493_full_batch(L, form):
    """The 4096-frame N=7493 batch on the persistent kernel (64 chunks), sampled."""
    w = I.make_workload("qc_n7493", frame_seed=9)
    p = dict(w.params, early_stop=0)
    h = L.Code.from_inputs(w.code)
    g = gpu_decode(h, w.code.n_vars, w.q0, L.make_params(form=form, kernel="persistent", **p))
    frames = np.array([0, 1, 63, 64, 2047, 4094, 4095])
    assert_int_parity({k: v[frames] for k, v in g.items()}, oracle_int(w.code, w.q0[frames], form, p))


def test_bounded_wait_gives_up_and_context_survives(L):
    assert L.ldpc_wait_selftest(0, 2000) == L.LDPC_ERR_TIMEOUT
    assert "gave up" in L.ldpc_last_error()
    # the context still decodes correctly afterwards
    w = I.make_workload("reg36_n1008", n_frames=9)
    h = L.Code.from_inputs(w.code)
    g = gpu_decode(h, w.code.n_vars, w.q0, L.make_params(form="ss_1bit", kernel="persistent", **w.params))
    assert_int_parity(g, oracle_int(w.code, w.q0, "ss_1bit", w.params))
