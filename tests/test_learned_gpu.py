"""GPU checks of the learned offset decoder and its training pieces against the
oracle: device AWGN generator, float32 forward, hand-written adjoint (against
the FP64 reverse-mode oracle and finite differences of the FP64 forward), BCE
loss, Adam, and the torch.autograd.Function wrapper."""
import numpy as np
import pytest

import oracle
from oracle import philox
from paper_cs_0609090_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_cs_0609090_gb300 import ldpc, learned
    w = I.make_workload("qc_n7493", n_frames=1, with_llr=False)
    return dict(torch=torch, ldpc=ldpc, learned=learned, code=w.code, h=ldpc.Code.from_inputs(w.code))


def _class_tab(code, beta_kc):
    deg = code.row_degrees()
    classes = sorted(set(deg.tolist()))
    return beta_kc[:, [classes.index(d) for d in deg]]


def test_device_awgn_matches_reference(env):
    torch, ldpc = env["torch"], env["ldpc"]
    N, F = 7493, 9
    llr = torch.empty((F, N), dtype=torch.float32, device="cuda")
    eb = torch.empty(F, dtype=torch.float32, device="cuda")
    ldpc.ldpc_awgn_llr_f32(N, 1234567, 1000, F, 1.5, 3.5, 0.593, None, llr, eb)
    ref, ref_eb = philox.awgn_llr(N, 1234567, 1000, F, 1.5, 3.5, 0.593)
    assert np.allclose(eb.cpu().numpy(), ref_eb, rtol=1e-6, atol=1e-6)
    got = llr.cpu().numpy()
    assert np.allclose(got, ref, rtol=2e-5, atol=2e-4), np.abs(got - ref).max()


def test_quantizer(env):
    torch, ldpc = env["torch"], env["ldpc"]
    x = np.array([-20.0, -1.0625, -0.0625, 0.0, 0.0624, 0.0625, 1.1875, 15.9, 16.0, 100.0], np.float32)
    q = torch.empty(x.size, dtype=torch.int8, device="cuda")
    ldpc.ldpc_quantize_llr(torch.from_numpy(x).cuda(), x.size, 0.125, 127, q)
    want = I.quantize(x.astype(np.float64), 0.125, 127)
    assert q.cpu().numpy().tolist() == want.tolist()


def _forward(env, q, beta_kc, K):
    torch, learned = env["torch"], env["learned"]
    dec = learned.LearnedDecoder(env["h"], K, q.shape[0])
    beta = torch.from_numpy(beta_kc.astype(np.float32)).cuda()
    z = dec.forward(torch.from_numpy(q.astype(np.float32)).cuda(), beta)
    return dec, beta, z


@pytest.mark.parametrize("ebn0", [2.0, 3.0])
def test_learned_forward_matches_fp64(env, ebn0):
    """Posteriors after 10 iterations against the FP64 oracle with the same
    per-iteration offsets.  Frames that decode are held to 1e-5 relative; at
    2.0 dB none does, and the offset rule amplifies float32 rounding on those
    oscillating trajectories (measured on this code: 8e-6 after 5 iterations,
    5e-4 after 12), so frames away from the decision threshold take 5e-4."""
    w = I.make_workload("qc_n7493", n_frames=16, ebn0_db=ebn0, zero_codeword=True)
    K = 10
    beta_kc = np.random.default_rng(2).uniform(0.1, 0.6, size=(K, 2))
    q = w.llr.astype(np.float32).astype(np.float64)
    _, _, z = _forward(env, q, beta_kc, K)
    o = oracle.decode_f64(w.code, q, form="ss_1bit", rule="offset", beta_tab=_class_tab(w.code, beta_kc),
                          max_iter=K, early_stop=0, want_margin=True)
    g = z.cpu().numpy()
    clean = o.margin > 1e-4
    err = np.abs(g - o.z) / np.maximum(1.0, np.abs(o.z))
    assert err[clean].max() <= 5e-4, err[clean].max()
    dec = clean & (o.ok == 1)
    if ebn0 >= 3.0:
        assert dec.sum() >= 12, dec.sum()
    if dec.any():
        assert err[dec].max() <= 1e-5, err[dec].max()


def _ref_class_grad(code, q, tab):
    loss_sum, db, gap = oracle.learned_grad(code, q, tab)
    deg = code.row_degrees()
    classes = sorted(set(deg.tolist()))
    return loss_sum, np.stack([db[:, deg == d].sum(axis=1) for d in classes], axis=1), gap


def test_learned_backward_matches_fp64_adjoint(env):
    """Channel values on a 1/4 grid and offsets on a 1/64 grid keep every forward
    quantity exactly representable in float32, so the GPU and the FP64 oracle take
    the same argmins, signs and offset branches (exact ties included, both with the
    lowest-position rule); the adjoints then differ only by float32 rounding."""
    w = I.make_workload("qc_n7493", n_frames=24, ebn0_db=2.5, zero_codeword=True)
    K = 10
    beta_kc = np.round(np.random.default_rng(5).uniform(0.1, 0.6, size=(K, 2)) * 64) / 64
    q = np.round(w.llr * 4) / 4
    F, N = q.shape
    loss_sum, ref, _ = _ref_class_grad(w.code, q, _class_tab(w.code, beta_kc))
    ref = ref / (F * N)
    dec, beta, z = _forward(env, q, beta_kc, K)
    zo = oracle.decode_f64(w.code, q, form="ss_1bit", rule="offset", beta_tab=_class_tab(w.code, beta_kc),
                           max_iter=K, early_stop=0).z
    assert np.array_equal(z.cpu().numpy().astype(np.float64), zo)      # the forward is exact
    loss = dec.loss(None, want_grad=True)
    got = dec.backward(beta, None).cpu().numpy()
    assert abs(float(loss.item()) - loss_sum / (F * N)) <= 1e-5 * loss_sum / (F * N)
    assert np.allclose(got, ref, rtol=1e-4, atol=1e-6 * np.abs(ref).max()), np.abs(got - ref).max()


def test_learned_backward_finite_differences(env):
    """Away from every kink (frames whose FP64 trajectory keeps each check's
    |u|, min2 - min1 and |min - beta| above 3e-4), the GPU adjoint equals central
    differences of the FP64 forward."""
    torch, learned, ldpc = env["torch"], env["learned"], env["ldpc"]
    w = I.make_workload("reg36_n1008", n_frames=256, ebn0_db=2.5, zero_codeword=True)
    K = 4
    beta_kc = np.random.default_rng(5).uniform(0.1, 0.6, size=(K, 1))
    tab = beta_kc[:, np.zeros(w.code.n_checks, int)]
    q = w.llr.astype(np.float32).astype(np.float64)
    _, _, gap = oracle.learned_grad(w.code, q, tab)
    q = q[gap > 3e-4]
    F, N = q.shape
    assert F >= 40
    h = ldpc.Code.from_inputs(w.code)
    dec = learned.LearnedDecoder(h, K, F)
    beta = torch.from_numpy(beta_kc.astype(np.float32)).cuda()
    dec.forward(torch.from_numpy(q.astype(np.float32)).cuda(), beta)
    dec.loss(None, want_grad=True)
    got = dec.backward(beta, None).cpu().numpy()
    eps = 1e-8
    for k in range(K):
        bp, bm = beta_kc.copy(), beta_kc.copy()
        bp[k, 0] += eps
        bm[k, 0] -= eps
        lp = np.logaddexp(0, -oracle.decode_f64(w.code, q, form="ss_1bit", rule="offset",
                                                beta_tab=bp[:, np.zeros(w.code.n_checks, int)], max_iter=K,
                                                early_stop=0).z).sum()
        lm = np.logaddexp(0, -oracle.decode_f64(w.code, q, form="ss_1bit", rule="offset",
                                                beta_tab=bm[:, np.zeros(w.code.n_checks, int)], max_iter=K,
                                                early_stop=0).z).sum()
        fd = (lp - lm) / (2 * eps) / (F * N)
        assert abs(got[k, 0] - fd) <= 1e-3 * abs(fd) + 1e-9, (k, got[k, 0], fd)


def test_autograd_function(env):
    torch, learned = env["torch"], env["learned"]
    w = I.make_workload("qc_n7493", n_frames=20, ebn0_db=2.5, zero_codeword=True)
    K = 5
    beta_kc = np.random.default_rng(9).uniform(0.1, 0.5, size=(K, 2))
    q = w.llr.astype(np.float32)
    dec = learned.LearnedDecoder(env["h"], K, q.shape[0])
    beta = torch.tensor(beta_kc, dtype=torch.float32, device="cuda", requires_grad=True)
    z = learned.LearnedOffsetDecode.apply(torch.from_numpy(q).cuda(), beta, dec)
    loss = torch.nn.functional.softplus(-z).mean()
    loss.backward()
    # the same gradient through the library's own loss kernel
    dec.forward(torch.from_numpy(q).cuda(), beta.detach())
    dec.loss(None, want_grad=True)
    direct = dec.backward(beta.detach(), None)
    assert torch.allclose(beta.grad, direct, rtol=1e-4, atol=1e-9)


def test_autograd_two_applies_then_backward_raises(env):
    """A decoder keeps the checkpoints of its latest forward only: the backward of
    an earlier apply must refuse to run on them, and one decoder per apply gives
    both gradients right."""
    torch, learned = env["torch"], env["learned"]
    code, h = env["code"], env["h"]
    w = I.make_workload("qc_n7493", n_frames=4, ebn0_db=2.5, zero_codeword=True)
    llr1 = torch.from_numpy(w.llr.astype(np.float32)).cuda()
    llr2 = torch.from_numpy((w.llr[::-1] * 0.9).astype(np.float32).copy()).cuda()
    dec = learned.LearnedDecoder(h, 3, 4)
    beta = torch.full((3, dec.C), 0.3, dtype=torch.float32, device="cuda", requires_grad=True)
    z1 = learned.LearnedOffsetDecode.apply(llr1, beta, dec)
    z2 = learned.LearnedOffsetDecode.apply(llr2, beta, dec)
    with pytest.raises(RuntimeError, match="no longer holds"):
        torch.autograd.grad(z1.sum(), beta, retain_graph=True)
    (g2,) = torch.autograd.grad(z2.sum(), beta)  # the latest apply is fine
    # two decoders: each backward matches its own single-apply gradient
    d1, d2 = learned.LearnedDecoder(h, 3, 4), learned.LearnedDecoder(h, 3, 4)
    a1 = learned.LearnedOffsetDecode.apply(llr1, beta, d1)
    a2 = learned.LearnedOffsetDecode.apply(llr2, beta, d2)
    (ga1,) = torch.autograd.grad(a1.sum(), beta)
    (ga2,) = torch.autograd.grad(a2.sum(), beta)
    solo = learned.LearnedDecoder(h, 3, 4)
    (gs1,) = torch.autograd.grad(learned.LearnedOffsetDecode.apply(llr1, beta, solo).sum(), beta)
    # (float atomics in the forward: equal up to rounding)
    assert torch.allclose(ga1, gs1, rtol=1e-4, atol=1e-6) and torch.allclose(ga2, g2, rtol=1e-4, atol=1e-6)


def test_adam_step(env):
    torch, ldpc = env["torch"], env["ldpc"]
    rng = np.random.default_rng(0)
    p, g = rng.normal(size=20).astype(np.float32), rng.normal(size=20).astype(np.float32)
    m, v = rng.normal(size=20).astype(np.float32) * 0.1, np.abs(rng.normal(size=20)).astype(np.float32) * 0.1
    tp, tg, tm, tv = (torch.from_numpy(x.copy()).cuda() for x in (p, g, m, v))
    ldpc.ldpc_adam_step(tp, tg, tm, tv, 20, 3, 0.01, 0.9, 0.999, 1e-8)
    m2 = 0.9 * m + 0.1 * g
    v2 = 0.999 * v + 0.001 * g * g
    p2 = p - 0.01 * (m2 / (1 - 0.9 ** 3)) / (np.sqrt(v2 / (1 - 0.999 ** 3)) + 1e-8)
    assert np.allclose(tp.cpu().numpy(), p2, rtol=1e-5, atol=1e-7)
    assert np.allclose(tm.cpu().numpy(), m2, rtol=1e-6) and np.allclose(tv.cpu().numpy(), v2, rtol=1e-6)


def test_training_reduces_loss(env):
    learned = env["learned"]
    res = learned.train(env["h"], K=5, total_frames=16 * 512, batch=512, lr=0.02)
    first, last = res["losses"][0][1], res["losses"][-1][1]
    assert np.isfinite(res["beta"]).all() and last < first
