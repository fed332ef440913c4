"""The float32 sum-product rule on the GPU (the accuracy reference of the
min-sum decoders): exact a-posteriori LLRs on cycle-free codes, parity with
the FP64 oracle's sum-product decoder, and fewer frame errors than min-sum on
the same frames."""
import numpy as np
import pytest

import oracle
from oracle import brute_force as bf
from paper_cs_0609090_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_cs_0609090_gb300 import ldpc
    return ldpc


def _spa(L, code, llr, max_iter, early_stop=0):
    import torch
    h = L.Code.from_inputs(code)
    p = L.make_params(dtype="f32", form="ss_fixed", rule="sum_product", max_iter=max_iter, early_stop=early_stop)
    bits, it, ok, z = L.decode(h, torch.from_numpy(np.ascontiguousarray(llr, dtype=np.float32)).cuda(), p,
                               want_llr=True)
    torch.cuda.synchronize()
    return dict(bits=L.unpack_bits(bits.cpu().numpy(), code.n_vars), iters=it.cpu().numpy(), ok=ok.cpu().numpy(),
                z=z.cpu().numpy())


@pytest.mark.parametrize("seed", range(6))
def test_tree_codes_reach_app_llr(L, seed):
    N = 8 + seed % 9
    code = I.tree_code(N, seed)
    cw = bf.codewords(N, [list(r) for r in code.rows()])
    q0 = np.random.default_rng(400 + seed).uniform(-1.5, 1.5, size=(40, N)).astype(np.float32)
    g = _spa(L, code, q0, 2 * N)
    app = bf.app_llr(cw, q0.astype(np.float64))
    assert np.allclose(g["z"], app, rtol=1e-4, atol=1e-4), np.abs(g["z"] - app).max()


def test_matches_fp64_oracle(L):
    """Frames whose FP64 trajectory keeps 1e-4 away from the decision threshold
    (295 of 300 at 3.0 dB): iterations, flags and decisions equal, posteriors of
    decoded frames within 1e-5 relative.  Measured without early stop on this
    code at 3.0 dB, the float32 posteriors of those frames stay within 4.5e-6 of
    FP64 at every iteration count up to 30."""
    w = I.make_workload("reg36_n1008", n_frames=300, ebn0_db=3.0)
    llr = w.llr.astype(np.float32)
    g = _spa(L, w.code, llr, 30, early_stop=1)
    o = oracle.decode_f64(w.code, llr.astype(np.float64), form="ss_fixed", rule="sum_product", max_iter=30,
                          early_stop=1, want_margin=True)
    clean = o.margin >= 1e-4
    assert clean.sum() >= 0.9 * clean.size, (~clean).sum()
    for key in ("iters", "ok", "bits"):
        assert np.array_equal(g[key][clean], o[key][clean]), key
    conv = clean & (o.ok == 1)
    assert conv.sum() >= 0.9 * clean.size
    err = np.abs(g["z"][conv] - o.z[conv]) / np.maximum(1.0, np.abs(o.z[conv]))
    assert err.max() <= 1e-5, err.max()


def test_fewer_frame_errors_than_min_sum(L):
    import torch
    w = I.make_workload("qc_n7493", n_frames=512, ebn0_db=2.5, frame_seed=13)
    g = _spa(L, w.code, w.llr, 30, early_stop=1)
    h = L.Code.from_inputs(w.code)
    bits, _, _, _ = L.decode(h, torch.from_numpy(w.q0).cuda(), L.make_params(**w.params))
    ms = L.unpack_bits(bits.cpu().numpy(), w.code.n_vars)
    fe_spa = int(np.any(g["bits"] != w.codewords, axis=1).sum())
    fe_ms = int(np.any(ms != w.codewords, axis=1).sum())
    assert fe_spa <= fe_ms, (fe_spa, fe_ms)


def test_rejected_outside_the_float_per_edge_path(L):
    import torch
    w = I.make_workload("reg36_n1008", n_frames=2)
    h = L.Code.from_inputs(w.code)
    for kw in (dict(dtype="int8"), dict(dtype="f32", form="ss_1bit")):
        with pytest.raises(L.LdpcError) as e:
            x = torch.from_numpy(w.q0).cuda()
            L.decode(h, x if kw["dtype"] == "int8" else x.float(), L.make_params(rule="sum_product", **kw))
        assert e.value.status == L.LDPC_ERR_UNSUPPORTED


def test_fer_tool_counts_errors_against_the_decoder_outputs(L):
    """paper_cs_0609090_gb300.fer on a few frames: its error count equals the
    count taken directly from the same decoder on the same device frames (random
    codewords of the code, each frame with its own noise)."""
    import torch
    from paper_cs_0609090_gb300 import fer as fer_mod
    w = I.make_workload("reg36_n1008", n_frames=1, with_llr=False)
    code = L.Code.from_inputs(w.code)
    rate = (w.code.n_vars - w.code.n_checks) / w.code.n_vars
    params = L.make_params(**w.params)
    pool = fer_mod.CodewordPool(w.code, 50, seed=3, device=torch.device("cuda"))
    run = fer_mod.int8_decoder(code, params, w.delta, w.qc, 128, torch.device("cuda"))
    r = fer_mod.run_point(run, w.code.n_vars, rate, 1.5, pool, min_errors=10 ** 9, max_frames=300, batch=128, seed=5)
    packed, cw = pool.rows(0, 300, torch.device("cuda"))
    llr = torch.empty((300, w.code.n_vars), dtype=torch.float32, device="cuda")
    L.ldpc_awgn_llr_f32(w.code.n_vars, 5, 0, 300, 1.5, 1.5, rate, packed, llr)
    q = torch.empty((300, w.code.n_vars), dtype=torch.int8, device="cuda")
    L.ldpc_quantize_llr(llr, 300 * w.code.n_vars, w.delta, w.qc, q)
    bits, iters, _, _ = L.decode(code, q, params)
    dec = L.unpack_bits(bits.cpu().numpy(), w.code.n_vars)
    assert r["frames"] == 300 and r["errors"] == int(np.any(dec != cw.cpu().numpy(), axis=1).sum())
    assert abs(r["mean_iters"] - float(iters.double().mean().item())) < 1e-9
    # every transmitted word is a codeword
    assert np.all(I.syndrome(w.code, cw.cpu().numpy()) == 0)
