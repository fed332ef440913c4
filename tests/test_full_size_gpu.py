"""Parity at the benchmarked sizes, in the launch configuration bench.py times:
the whole batch is decoded on the GPU and the oracle checks sampled frames
spread over the batch (first and last frame pairs, the ragged tail, random
ones).  Also the empty batch and a batch four times the benchmarked one."""
import numpy as np
import pytest

import oracle
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


def _sample(F, k, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, 1, F // 2, F - 2, F - 1], rng.choice(F, k, replace=False)]))


@pytest.mark.parametrize("form", FORMS_INT)
def test_irr_64800_full_batch_sampled(L, form):
    """1024 frames, 50 iterations, early stop off: the library's choice (as
    bench.py times it), the two-launch and the persistent streaming kernels,
    sampled frames against the oracle."""
    w = I.make_workload("irr_n64800")
    p = dict(w.params, early_stop=0)
    h = L.Code.from_inputs(w.code)
    frames = _sample(w.n_frames, 3, 1)
    o = oracle_int(w.code, w.q0[frames], form, p)
    for kern in ("auto", "stream", "persistent"):
        g = gpu_decode(h, w.code.n_vars, w.q0, L.make_params(form=form, kernel=kern, **p))
        assert_int_parity({k: v[frames] for k, v in g.items()}, o)


def test_irr_64800_f32_full_batch_sampled(L):
    """The float32 normalized path on the whole 1024-frame batch; sampled frames
    against the FP64 oracle: posteriors within 1e-5 relative (the normalized rule
    contracts rounding errors), decisions equal wherever |Z| > 1e-3."""
    import torch
    w = I.make_workload("irr_n64800")
    h = L.Code.from_inputs(w.code)
    params = L.make_params(dtype="f32", form="ss_1bit", rule="normalized", norm_f32=0.75, max_iter=50,
                           early_stop=0)
    t = torch.from_numpy(w.llr.astype(np.float32)).cuda()
    bits, iters, ok, z = L.decode(h, t, params, want_llr=True)
    torch.cuda.synchronize()
    frames = _sample(w.n_frames, 2, 2)
    q = w.llr[frames].astype(np.float32).astype(np.float64)
    o = oracle.decode_f64(w.code, q, form="ss_1bit", rule="normalized", lam=0.75, max_iter=50, early_stop=0)
    gz = z.cpu().numpy()[frames]
    err = np.abs(gz - o.z) / np.maximum(1.0, np.abs(o.z))
    assert err.max() <= 1e-5, err.max()
    gb = L.unpack_bits(bits.cpu().numpy(), w.code.n_vars)[frames]
    nz = np.abs(o.z) > 1e-3
    assert np.array_equal(gb[nz], o.bits[nz])
    assert np.all(iters.cpu().numpy() == 50)


@pytest.mark.parametrize("form", FORMS_INT)
def test_multi8_full_batch_sampled(L, form):
    """The whole eight-code batch (Poisson(512) frames per code) in the plan
    bench.py replays; three frames per code checked."""
    import torch
    ws = I.make_multi_workload()
    for w in ws:
        w.params["early_stop"] = 0
    codes = [L.Code.from_inputs(w.code) for w in ws]
    llrs = [torch.from_numpy(w.q0).cuda() for w in ws]
    mb = L.MultiBatch(codes, llrs, [L.make_params(form=form, **w.params) for w in ws])
    mb.decode()
    torch.cuda.synchronize()
    for j, w in enumerate(ws):
        frames = np.array([0, w.n_frames - 1, int(np.random.default_rng(j).integers(1, w.n_frames - 1))])
        bits, iters, ok, _ = mb.outputs[j]
        g = dict(bits=L.unpack_bits(bits.cpu().numpy(), w.code.n_vars)[frames], iters=iters.cpu().numpy()[frames],
                 ok=ok.cpu().numpy()[frames])
        try:
            assert_int_parity(g, oracle_int(w.code, w.q0[frames], form, w.params))
        except AssertionError as e:
            raise AssertionError(f"{w.name}: {e}")


def test_zero_frames_is_a_noop(L):
    import torch
    w = I.make_workload("qc_n7493", n_frames=2)
    h = L.Code.from_inputs(w.code)
    bits = torch.full((2, (w.code.n_vars + 7) // 8), 0xAB, dtype=torch.uint8, device="cuda")
    it = torch.full((2,), -7, dtype=torch.int32, device="cuda")
    ok = torch.full((2,), 9, dtype=torch.uint8, device="cuda")
    q = torch.from_numpy(w.q0).cuda()
    for kern in ("auto", "onchip_int", "stream", "cluster", "persistent", "pingpong"):
        p = L.make_params(kernel=kern, **w.params)
        assert L.ldpc_workspace_size(h.handle, p, 0) == 0
        L.ldpc_decode_batch(h.handle, p, q, 0, bits, it, ok)
    torch.cuda.synchronize()
    assert int(bits.min()) == 0xAB and int(it.max()) == -7 and int(ok.min()) == 9


@pytest.mark.parametrize("form", FORMS_INT)
def test_qc_7493_four_times_the_batch(L, form):
    """16384 frames (four times the benchmarked batch, 123 MB of LLRs): the
    persistent grid loops over 8192 frame pairs; sampled frames."""
    w = I.make_workload("qc_n7493", n_frames=16384, frame_seed=5)
    p = dict(w.params, early_stop=0)
    h = L.Code.from_inputs(w.code)
    g = gpu_decode(h, w.code.n_vars, w.q0, L.make_params(form=form, **p), want_llr=False)
    frames = _sample(w.n_frames, 6, 3)
    assert_int_parity({k: v[frames] for k, v in g.items()}, oracle_int(w.code, w.q0[frames], form, p))
