"""ldpc_decode_batch inside a CUDA graph: every kernel path is captured once
(after one eager call on the device, as the header requires) and replayed on
new channel values written into the same input buffer; the outputs equal the
oracle's for the new values."""
import numpy as np
import pytest

import oracle
from paper_cs_0609090_gb300 import inputs as I
from gpu_helpers import assert_int_parity, oracle_int

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_cs_0609090_gb300 import ldpc
    return ldpc


CASES = [("reg36_n1008", dict(form="ss_1bit")), ("reg36_n1008", dict(form="ss_fixed")),
         ("reg36_n1008", dict(form="two_scan")), ("reg36_n1008", dict(form="ss_1bit", kernel="stream")),
         ("reg36_n1008", dict(form="ss_fixed", kernel="onchip_int")),
         ("reg36_n1008", dict(form="ss_1bit", schedule="layered")),
         ("qc_n7493", dict(form="ss_1bit", kernel="cluster"))]


@pytest.mark.parametrize("name,kw", CASES, ids=[f"{c[0]}-" + "-".join(c[1].values()) for c in CASES])
def test_decode_batch_replays_from_a_graph(L, name, kw):
    import torch
    F = 24
    w = I.make_workload(name, n_frames=F, ebn0_db=2.0, frame_seed=3)
    p = dict(w.params)
    h = L.Code.from_inputs(w.code)
    params = L.make_params(**dict(p, **kw))
    N = w.code.n_vars
    q = torch.from_numpy(w.q0).cuda()
    bits = torch.zeros((F, (N + 7) // 8), dtype=torch.uint8, device="cuda")
    it = torch.zeros(F, dtype=torch.int32, device="cuda")
    ok = torch.zeros(F, dtype=torch.uint8, device="cuda")
    z = torch.zeros((F, N), dtype=torch.int16, device="cuda")
    wsb = L.ldpc_workspace_size(h.handle, params, F)
    ws = torch.empty(wsb + 256, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) & ~255

    class W:
        def data_ptr(self):
            return base
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())

    def call():
        L.ldpc_decode_batch(h.handle, params, q, F, bits, it, ok, z, W() if wsb else None, wsb, s)
    with torch.cuda.stream(s):
        call()                                   # eager first call on the device
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        call()
    for seed in (11, 12):
        w2 = I.make_workload(name, n_frames=F, ebn0_db=2.0, frame_seed=seed)
        q.copy_(torch.from_numpy(w2.q0))
        bits.zero_(), it.fill_(-1), ok.fill_(7), z.zero_()
        g.replay()
        torch.cuda.synchronize()
        got = dict(bits=L.unpack_bits(bits.cpu().numpy(), N), iters=it.cpu().numpy(), ok=ok.cpu().numpy(),
                   z=z.cpu().numpy())
        form = kw["form"]
        if kw.get("schedule") == "layered":
            lay = L.ldpc_code_layers(h.handle, w.code.n_checks)[1]
            ref = oracle.decode_layered_int(w.code, w2.q0.astype(np.int32), lay, rule=p["rule"],
                                            offset=p.get("offset", 0), msg_sat=p["msg_sat"],
                                            max_iter=p["max_iter"], early_stop=p["early_stop"])
        else:
            ref = oracle_int(w.code, w2.q0, form, p)
        assert_int_parity(got, ref)
