"""Guard bands around every buffer a decode writes (canaries, in place of a
memory checker): each output and the workspace sit inside a larger allocation
whose 4 KiB before and after hold a fixed byte pattern, the workspace given at
exactly the size the library asks for.  After the decode the bands must be
unchanged and the results equal an unguarded decode.  Frame counts are ragged
(odd, not multiples of the 32- or 64-frame lane groups) so that the tails of
every lane mapping are exercised.  This catches writes past the end or before
the start of any buffer, the typical mistake of a tail or offset computation."""
import ctypes

import numpy as np
import pytest

from paper_cs_0609090_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GUARD = 4096
PATTERN = 0xA5


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_cs_0609090_gb300 import ldpc
    return ldpc


class Guarded:
    """nbytes usable bytes at a 4 KiB-aligned offset inside a pattern-filled
    allocation."""

    def __init__(self, nbytes):
        import torch
        self.n = int(nbytes)
        self.big = torch.full((2 * GUARD + max(self.n, 1) + 4096,), PATTERN, dtype=torch.uint8, device="cuda")
        base = self.big.data_ptr()
        self.off = ((base + GUARD + 4095) & ~4095) - base
        self.ptr = base + self.off

    def view(self, dtype, shape):
        import torch
        t = self.big[self.off:self.off + self.n].view(dtype)
        return t.view(shape)

    def intact(self):
        b = self.big.cpu().numpy()
        return bool(np.all(b[:self.off] == PATTERN) and np.all(b[self.off + self.n:] == PATTERN))


def _decode_guarded(L, h, q, params, F, N):
    import torch
    out_dtype = torch.int16 if params.dtype == L.LDPC_DTYPE_INT8 else torch.float32
    esz = 2 if params.dtype == L.LDPC_DTYPE_INT8 else 4
    gb, gi, go, gz = Guarded(F * ((N + 7) // 8)), Guarded(4 * F), Guarded(F), Guarded(esz * F * N)
    ws_bytes = L.ldpc_workspace_size(h.handle, params, F)
    gw = Guarded(ws_bytes) if ws_bytes else None
    P = ctypes.c_void_p
    L._check(L._lib.ldpc_decode_batch(P(h.handle), ctypes.byref(params), P(q.data_ptr()), F, P(gb.ptr), P(gi.ptr),
                                      P(go.ptr), P(gz.ptr), P(gw.ptr) if gw else None, ws_bytes,
                                      L._stream_handle(None)), "ldpc_decode_batch")
    torch.cuda.synchronize()
    for name, g in (("bits", gb), ("iters", gi), ("ok", go), ("llr_out", gz), ("workspace", gw)):
        if g is not None:
            assert g.intact(), f"{name}: a guard band was written"
    return (gb.view(torch.uint8, (F, (N + 7) // 8)).cpu().numpy(), gi.view(torch.int32, (F,)).cpu().numpy(),
            go.view(torch.uint8, (F,)).cpu().numpy(), gz.view(out_dtype, (F, N)).cpu().numpy())


def _check_family(L, w, F, kw, f32=False):
    import torch
    h = L.Code.from_inputs(w.code)
    src = w.llr.astype(np.float32) if f32 else w.q0
    q = torch.from_numpy(np.ascontiguousarray(src[:F])).cuda()
    params = L.make_params(**dict(w.params, **kw))
    got = _decode_guarded(L, h, q, params, F, w.code.n_vars)
    bits, it, ok, z = L.decode(h, q, params, want_llr=True)
    torch.cuda.synchronize()
    ref = (bits.cpu().numpy(), it.cpu().numpy(), ok.cpu().numpy(), z.cpu().numpy())
    for a, b, name in zip(got, ref, ("bits", "iters", "ok", "llr_out")):
        if f32 and name == "llr_out":
            continue  # float atomics: the summation order may differ between the two runs
        assert np.array_equal(a, b), name


CASES = [
    ("qc_n7493", {"kernel": "onchip_half"}),
    ("qc_n7493", {"kernel": "onchip_int"}),
    ("qc_n7493", {"kernel": "stream"}),
    ("qc_n7493", {"kernel": "persistent"}),
    ("qc_n7493", {"form": "two_scan"}),
    ("qc_n7493", {"form": "two_scan", "kernel": "stream"}),
    ("qc_n7493", {"form": "two_scan_1bit"}),
    ("qc_n7493", {"schedule": "layered"}),
    ("qc_n7493", {"posterior": "sat8", "kernel": "stream"}),
    ("reg36_n1008", {"kernel": "pingpong"}),
    ("reg36_n1008", {"kernel": "onchip_half", "form": "ss_fixed"}),
    ("irr_n64800", {"kernel": "cluster"}),
    ("irr_n64800", {"kernel": "pingpong", "form": "ss_fixed"}),
]


@pytest.mark.parametrize("F", [1, 67])
@pytest.mark.parametrize("wl,kw", CASES, ids=[f"{w}-{'-'.join(f'{k}={v}' for k, v in kw.items())}" for w, kw in CASES])
def test_guard_bands_int8(L, wl, kw, F):
    w = I.make_workload(wl, n_frames=67, frame_seed=9)
    _check_family(L, w, F, dict(kw, max_iter=4, early_stop=1))


@pytest.mark.parametrize("F", [1, 67])
@pytest.mark.parametrize("form", ["ss_1bit", "ss_fixed"])
def test_guard_bands_f32(L, form, F):
    w = I.make_workload("reg36_n1008", n_frames=67, frame_seed=9)
    _check_family(L, w, F, dict(dtype="f32", form=form, rule="normalized", norm_f32=0.75, max_iter=6), f32=True)


def test_guard_bands_multi_and_learned(L):
    """The eight-code batch (outputs of every job guarded) and the learned
    forward (posteriors and checkpoint workspace guarded)."""
    import torch
    ws_list = I.make_multi_workload(frames=[33, 17, 5, 41, 9, 3, 12, 7])
    codes = [L.Code.from_inputs(w.code) for w in ws_list]
    guards, jobs = [], []
    for c, w in zip(codes, ws_list):
        F, N = w.q0.shape
        q = torch.from_numpy(w.q0).cuda()
        g = [Guarded(F * ((N + 7) // 8)), Guarded(4 * F), Guarded(F), Guarded(2 * F * N)]
        guards.append((q, g))
        p = L.make_params(**dict(w.params, max_iter=3))
        jobs.append(L.ldpc_multi_job(c.handle, p, q.data_ptr(), F, g[0].ptr, g[1].ptr, g[2].ptr, g[3].ptr))
    plan = L.ldpc_multi_create(jobs)
    try:
        wsb = L.ldpc_multi_workspace_size(plan)
        gw = Guarded(wsb) if wsb else None
        L._check(L._lib.ldpc_multi_decode(ctypes.c_void_p(plan), ctypes.c_void_p(gw.ptr) if gw else None, wsb,
                                          L._stream_handle(None)), "ldpc_multi_decode")
        torch.cuda.synchronize()
        for j, (_, g) in enumerate(guards):
            assert all(x.intact() for x in g), f"job {j}: a guard band was written"
        assert gw is None or gw.intact()
    finally:
        L.ldpc_multi_destroy(plan)

    w = I.make_workload("qc_n7493", n_frames=37, frame_seed=2)
    h = L.Code.from_inputs(w.code)
    K, F, N = 4, 37, w.code.n_vars
    n_cls = 2
    beta = torch.full((K, n_cls), 0.3, dtype=torch.float32, device="cuda")
    llr = torch.from_numpy(w.llr.astype(np.float32)).cuda()
    wsb = L.ldpc_learned_workspace_size(h.handle, K, F)
    gz, gw = Guarded(4 * F * N), Guarded(wsb)
    L._check(L._lib.ldpc_learned_forward(ctypes.c_void_p(h.handle), K, ctypes.c_void_p(beta.data_ptr()),
                                         ctypes.c_void_p(llr.data_ptr()), F, ctypes.c_void_p(gz.ptr),
                                         ctypes.c_void_p(gw.ptr), wsb, L._stream_handle(None)),
             "ldpc_learned_forward")
    torch.cuda.synchronize()
    assert gz.intact() and gw.intact()
