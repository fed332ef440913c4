"""ldpc_decode_batch_noalloc: decoding for callers that cannot allocate device
memory (the library's built-in device scratch replaces the caller's workspace).

Checked through the C ABI against ldpc_decode_batch on the same inputs, with two
calls in a row so that whatever the first call leaves in the shared scratch
cannot leak into the second.  Named test_zz_* so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_cs_0609090_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_cs_0609090_gb300 import ldpc
    return ldpc


def _outputs(torch, F, N, llr_dtype):
    return (torch.empty((F, (N + 7) // 8), dtype=torch.uint8, device="cuda"),
            torch.empty(F, dtype=torch.int32, device="cuda"),
            torch.empty(F, dtype=torch.uint8, device="cuda"),
            torch.empty((F, N), dtype=llr_dtype, device="cuda"))


def _compare(L, code, q_host, params):
    """Decode with the no-allocation entry point and with ldpc_decode_batch
    (streaming kernel, caller workspace); return both results on the host."""
    import torch
    F, N = q_host.shape
    q = torch.from_numpy(q_host).cuda()
    a = _outputs(torch, F, N, torch.int16)
    L.ldpc_decode_batch_noalloc(code.handle, params, q, F, *a)
    ref_params = L.make_params(form=params.form, rule=params.rule, offset=params.offset,
                               norm_num=params.norm_num, norm_shift=params.norm_shift, msg_sat=params.msg_sat,
                               max_iter=params.max_iter, early_stop=params.early_stop, kernel="stream")
    b = _outputs(torch, F, N, torch.int16)
    need = L.ldpc_workspace_size(code.handle, ref_params, F)
    ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")

    class _Ptr:
        def data_ptr(self):
            return (ws.data_ptr() + 255) & ~255
    L.ldpc_decode_batch(code.handle, ref_params, q, F, *b, workspace=_Ptr(), ws_bytes=need)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in a], [t.cpu().numpy() for t in b]


@pytest.mark.parametrize("form", ["ss_1bit", "ss_fixed"])
def test_noalloc_matches_decode_batch_twice(L, form):
    w = I.make_workload("qc_n7493", n_frames=96, ebn0_db=2.0)
    code = L.Code.from_inputs(w.code)
    params = L.make_params(form=form, **w.params)
    # two calls in a row on different frames: the second must not see the first's scratch
    for q in (w.q0[:96], w.q0[40:75]):
        got, ref = _compare(L, code, np.ascontiguousarray(q), params)
        for x, y in zip(got, ref):
            assert np.array_equal(x, y)


def test_noalloc_large_code_and_size_limit(L):
    import torch
    w = I.make_workload("irr_n64800", n_frames=64, frame_seed=5)
    code = L.Code.from_inputs(w.code)
    params = L.make_params(**w.params)
    for F in (64, 9):
        got, ref = _compare(L, code, np.ascontiguousarray(w.q0[:F]), params)
        for x, y in zip(got, ref):
            assert np.array_equal(x, y)
    # 128 frames of this code need more scratch than the library holds
    q = torch.zeros((128, w.code.n_vars), dtype=torch.int8, device="cuda")
    with pytest.raises(L.LdpcError) as e:
        L.ldpc_decode_batch_noalloc(code.handle, params, q, 128, *_outputs(torch, 128, w.code.n_vars, torch.int16))
    assert e.value.status == L.LDPC_ERR_UNSUPPORTED
    assert "static scratch holds" in str(e.value)
