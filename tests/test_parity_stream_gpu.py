"""GPU vs oracle parity of the device-memory (streaming) decoders: the int8 path
(bit-exact, packed binary16 lanes) and the float32 path (within tolerance of the
FP64 oracle; float atomics make the summation order vary)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_cs_0609090_gb300 import inputs as I
from gpu_helpers import FORMS_INT, assert_int_parity, gpu_decode, oracle_int

pytestmark = pytest.mark.gpu

# |Z_gpu - Z_fp64| <= RTOL * max(1, |Z_fp64|).  The normalized rule (lambda < 1)
# scales every rounding error down at each check, so RTOL holds for every frame
# after 30 iterations (measured 8.7e-6 on the N=1008 code at 2.0 dB).  The offset
# rule has no such contraction: while a frame has not reached a codeword its
# oscillating trajectory amplifies the rounding error about tenfold every four
# iterations (N=7493 at 2.5 dB, offset 0.5: 6e-7 after 1, 8e-6 after 5, 5e-4 after
# 12, 9e-2 after 20; N=1008 at 2.0 dB: 6.1e-6 after 12, 5e-5 after 20), and a frame
# that decodes late keeps what it gathered (1.2e-4 measured).  Offset frames that
# stop within OFFSET_TIGHT_ITERS iterations are held to RTOL, later ones and the
# 12-iteration all-frames check to RTOL_OFFSET.
RTOL = 1e-5
RTOL_OFFSET = 5e-4
OFFSET_TIGHT_ITERS = 10


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_cs_0609090_gb300 import ldpc
    return ldpc


def _int(L, code, q0, form, p, kernel="stream"):
    h = L.Code.from_inputs(code)
    g = gpu_decode(h, code.n_vars, q0, L.make_params(form=form, kernel=kernel, **p))
    assert_int_parity(g, oracle_int(code, q0, form, p))
    return g


STREAM_KERNELS = ("stream", "persistent", "pingpong")


@pytest.mark.parametrize("kernel", STREAM_KERNELS)
@pytest.mark.parametrize("form", FORMS_INT)
@pytest.mark.parametrize("early_stop", [1, 0])
def test_int8_stream_small_codes(L, form, early_stop, kernel):
    """301 frames of the N=1008 code: 151 frame pairs, 5 chunks of 32 pairs, so
    the persistent decoder runs two full groups of two chunks and a last group of
    one, with a ragged last chunk and an odd frame count."""
    w = I.make_workload("reg36_n1008", n_frames=301, ebn0_db=1.8)
    _int(L, w.code, w.q0, form, dict(w.params, early_stop=early_stop), kernel=kernel)
    w = I.make_workload("qc_n7493", n_frames=67, ebn0_db=2.0)
    if kernel == "pingpong":  # checks of degree 14 and 15: the ping-pong kernel takes degree <= 8
        h = L.Code.from_inputs(w.code)
        with pytest.raises(L.LdpcError):
            L.ldpc_workspace_size(h.handle, L.make_params(form=form, kernel=kernel, **w.params), 67)
        return
    _int(L, w.code, w.q0, form, dict(w.params, early_stop=early_stop), kernel=kernel)


@pytest.mark.parametrize("kernel", STREAM_KERNELS)
@pytest.mark.parametrize("form", FORMS_INT)
def test_int8_stream_edge_cases(L, form, kernel):
    w = I.make_workload("reg36_n1008", n_frames=65, ebn0_db=1.0)
    for F in (1, 2, 33, 65):
        _int(L, w.code, w.q0[:F], form, w.params, kernel=kernel)
    _int(L, w.code, w.q0[:5], form, dict(w.params, max_iter=0), kernel=kernel)
    _int(L, w.code, w.q0[:5], form, dict(w.params, max_iter=1), kernel=kernel)
    _int(L, w.code, w.q0[:5], form, dict(w.params, max_iter=0, early_stop=0), kernel=kernel)
    g = _int(L, w.code, I.noiseless(w.codewords, 31), form, w.params, kernel=kernel)
    assert np.all(g["iters"] == 0)


@pytest.mark.parametrize("form", FORMS_INT)
@pytest.mark.parametrize("early_stop", [1, 0])
def test_int8_irregular_64800(L, form, early_stop):
    """The N=64800 code does not fit one SM: the ping-pong kernel (the library's
    choice), the two-launch streaming kernel, the persistent kernel and the
    cluster kernel (8 CTAs, distributed shared memory) all decode it."""
    w = I.make_workload("irr_n64800", n_frames=7, frame_seed=3)
    p = dict(w.params, early_stop=early_stop)
    h = L.Code.from_inputs(w.code)
    assert L.ldpc_workspace_size(h.handle, L.make_params(form=form, **p), 7) > 0
    for kern in ("auto", "pingpong", "persistent", "stream", "cluster"):
        _int(L, w.code, w.q0, form, p, kernel=kern)
        if early_stop:
            q = I.noiseless(w.codewords[:2], 127)
            g = _int(L, w.code, q, form, p, kernel=kern)
            assert np.all(g["iters"] == 0)


def _f32(L, code, llr, form, rule, lam=0.75, offset=0.0, max_iter=50, early_stop=0, kernel="stream"):
    import torch
    h = L.Code.from_inputs(code)
    params = L.make_params(dtype="f32", form=form, rule=rule, norm_f32=lam, offset_f32=offset,
                           max_iter=max_iter, early_stop=early_stop, kernel=kernel)
    t = torch.from_numpy(np.ascontiguousarray(llr, dtype=np.float32)).cuda()
    bits, iters, ok, z = L.decode(h, t, params, want_llr=True)
    torch.cuda.synchronize()
    g = dict(bits=L.unpack_bits(bits.cpu().numpy(), code.n_vars), iters=iters.cpu().numpy(),
             ok=ok.cpu().numpy(), z=z.cpu().numpy())
    o = oracle.decode_f64(code, llr.astype(np.float32).astype(np.float64), form=form, rule=rule, lam=lam,
                          offset=offset, max_iter=max_iter, early_stop=early_stop, want_margin=True)
    return g, o


def test_f32_hamming_golden(L):
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hamming74_min_sum.json")))
    code = I.from_rows(7, gold["code"]["rows"])
    q = np.array([gold["q0"]] * 3, dtype=np.float64)
    for form in FORMS_INT:
        g, _ = _f32(L, code, q, form, "normalized", max_iter=1)
        assert g["z"][0].tolist() == gold["normalized_float_0p75"]["Z1"]
        g, _ = _f32(L, code, q, form, "plain", max_iter=2)
        assert g["z"][0].tolist() == gold["plain"]["Z2"]


@pytest.mark.parametrize("form", FORMS_INT)
def test_f32_irregular_64800_normalized(L, form):
    w = I.make_workload("irr_n64800", n_frames=5, frame_seed=7)
    g, o = _f32(L, w.code, w.llr, form, "normalized", max_iter=50, kernel="auto")
    err = np.abs(g["z"] - o.z) / np.maximum(1.0, np.abs(o.z))
    assert err.max() <= RTOL, f"max relative error {err.max():.3g}"
    assert np.array_equal(g["iters"], o.iters)
    nz = np.abs(o.z) > 1e-3
    assert np.array_equal(g["bits"][nz], o.bits[nz])


# Frames whose FP64 posteriors come within this distance of the decision rule
# (min over iterations of |Z_n|) may legitimately stop at another iteration or
# decide a bit differently under float32 rounding.
MARGIN = 1e-4


@pytest.mark.parametrize("form", FORMS_INT)
@pytest.mark.parametrize("rule,offset", [("offset", 0.5), ("normalized", 0.0)])
def test_f32_early_stop_regular(L, form, rule, offset):
    """Frames away from the decision boundary: iteration counts, flags and
    decisions equal the FP64 oracle's.  Frames the oracle decodes to a codeword
    have posteriors within RTOL (under the offset rule: those that stop within
    OFFSET_TIGHT_ITERS iterations; later ones within RTOL_OFFSET); frames that
    run to the cap without one are excluded from that check."""
    w = I.make_workload("reg36_n1008", n_frames=400, ebn0_db=2.0)
    g, o = _f32(L, w.code, w.llr, form, rule, offset=offset, max_iter=30, early_stop=1)
    clean = o.margin >= MARGIN
    assert clean.sum() >= 0.9 * clean.size, f"{(~clean).sum()} near-tie frames"
    assert np.array_equal(g["iters"][clean], o.iters[clean])
    assert np.array_equal(g["ok"][clean], o.ok[clean])
    assert np.array_equal(g["bits"][clean], o.bits[clean])
    conv = clean & (o.ok == 1)
    assert conv.sum() >= 0.8 * clean.size
    err = np.abs(g["z"] - o.z) / np.maximum(1.0, np.abs(o.z))
    tight = conv & (o.iters <= OFFSET_TIGHT_ITERS) if rule == "offset" else conv
    assert tight.sum() >= 0.5 * clean.size
    assert err[tight].max() <= RTOL, f"max relative error {err[tight].max():.3g}"
    assert err[conv].max() <= RTOL_OFFSET, f"max relative error {err[conv].max():.3g}"


def _clean_parity(g, o, rtol, min_clean=0.9):
    """Iterations, flags and decisions equal on the frames away from the decision
    boundary; posteriors of the decoded ones within rtol of the FP64 oracle."""
    clean = o.margin >= MARGIN
    assert clean.sum() >= min_clean * clean.size, f"{(~clean).sum()} near-tie frames"
    for key in ("iters", "ok", "bits"):
        assert np.array_equal(g[key][clean], o[key][clean]), key
    conv = clean & (o.ok == 1)
    if conv.any():
        err = np.abs(g["z"][conv] - o.z[conv]) / np.maximum(1.0, np.abs(o.z[conv]))
        assert err.max() <= rtol, f"max relative error {err.max():.3g}"
    return clean


@pytest.mark.parametrize("form", FORMS_INT)
def test_f32_edge_cases(L, form):
    """One frame and ragged frame counts (the lanes of the last warp partly
    empty), max_iter = 0 (the channel values returned as they are), and noiseless
    frames (stopped at iteration 0 from the first posterior buffer)."""
    w = I.make_workload("reg36_n1008", n_frames=65, ebn0_db=2.0, frame_seed=5)
    for F in (1, 33, 65):
        g, o = _f32(L, w.code, w.llr[:F], form, "normalized", max_iter=30, early_stop=1)
        _clean_parity(g, o, RTOL, min_clean=0.8)
    g, o = _f32(L, w.code, w.llr[:7], form, "normalized", max_iter=0, early_stop=1)
    assert np.array_equal(g["z"], w.llr[:7].astype(np.float32))
    assert np.all(g["iters"] == 0)
    assert np.array_equal(g["ok"], o.ok) and np.array_equal(g["bits"], o.bits)
    q = I.noiseless(w.codewords[:3], 31).astype(np.float32)
    g, o = _f32(L, w.code, q, form, "normalized", max_iter=30, early_stop=1)
    assert np.all(g["iters"] == 0) and np.all(g["ok"] == 1) and np.array_equal(g["z"], q)


@pytest.mark.parametrize("form", FORMS_INT)
def test_f32_other_degrees(L, form):
    """Row degree 9 (the kernel's loop body) and the quasi-cyclic code's degrees
    14 / 15 (unrolled bodies in the Section V form), with frames stopping at odd
    and even iteration counts, whose results come from different posterior
    buffers."""
    code = I.regular_code(990, 3, 9, seed=5)
    zero = np.zeros((160, code.n_vars), np.uint8)
    llr = I.awgn_llr(zero, 3.2, 2.0 / 3.0, seed=17)
    g, o = _f32(L, code, llr, form, "normalized", max_iter=25, early_stop=1)
    clean = _clean_parity(g, o, RTOL, min_clean=0.8)
    assert len(set((g["iters"][clean] % 2).tolist())) == 2
    w = I.make_workload("qc_n7493", n_frames=96, ebn0_db=3.3, frame_seed=6)
    g, o = _f32(L, w.code, w.llr, form, "normalized", max_iter=25, early_stop=1)
    clean = _clean_parity(g, o, RTOL, min_clean=0.8)
    assert len(set((g["iters"][clean] % 2).tolist())) == 2
    g, o = _f32(L, w.code, w.llr[:40], form, "offset", offset=0.25, max_iter=12, early_stop=0)
    err = np.abs(g["z"] - o.z) / np.maximum(1.0, np.abs(o.z))
    assert err.max() <= RTOL_OFFSET, f"max relative error {err.max():.3g}"


def test_stream_workspace_contract(L):
    import torch
    w = I.make_workload("irr_n64800", n_frames=2)
    h = L.Code.from_inputs(w.code)
    params = L.make_params(kernel="stream", **w.params)
    need = L.ldpc_workspace_size(h.handle, params, 2)
    assert need > 0
    q = torch.from_numpy(w.q0).cuda()
    bits = torch.empty((2, (w.code.n_vars + 7) // 8), dtype=torch.uint8, device="cuda")
    it = torch.empty(2, dtype=torch.int32, device="cuda")
    ok = torch.empty(2, dtype=torch.uint8, device="cuda")
    ws = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) & ~255

    class P:
        def __init__(self, v):
            self.v = v

        def data_ptr(self):
            return self.v
    with pytest.raises(L.LdpcError) as e:        # too small
        L.ldpc_decode_batch(h.handle, params, q, 2, bits, it, ok, None, P(base), need - 1)
    assert e.value.status == L.LDPC_ERR_INVALID_ARG
    with pytest.raises(L.LdpcError) as e:        # misaligned
        L.ldpc_decode_batch(h.handle, params, q, 2, bits, it, ok, None, P(base + 16), need)
    assert e.value.status == L.LDPC_ERR_INVALID_ARG
    L.ldpc_decode_batch(h.handle, params, q, 2, bits, it, ok, None, P(base), need)
    torch.cuda.synchronize()


def _mixed_rows(n_vars, n_checks, dmin, dmax, seed):
    """Rows of degrees dmin..dmax on random distinct variables, every variable
    in at least one check, ordered so that warps of four checks mix degrees."""
    rng = np.random.default_rng(seed)
    rows = [sorted(rng.choice(n_vars, size=int(rng.integers(dmin, dmax + 1)), replace=False).tolist())
            for _ in range(n_checks)]
    seen = {v for r in rows for v in r}
    for v in range(n_vars):
        if v not in seen:
            r = rows[int(rng.integers(n_checks))]
            if len(r) < dmax:
                r.append(v)
                r.sort()
            else:
                rows.append([v, (v + 1) % n_vars])
    return rows


@pytest.mark.parametrize("dmax", [7, 8])
@pytest.mark.parametrize("form", FORMS_INT)
def test_pingpong_mixed_degrees(L, form, dmax):
    """The ping-pong decoder on codes of row degrees 2 to 7 or 8: mixed degrees
    in a warp's checks and uniform degrees other than 6 and 7 (the unstaged
    path) and uniform runs of 6 and 7 (the staged path), against the oracle
    under every rule, with and without early stop, with a small Qm (both minima
    saturated) and the largest, on random LLRs."""
    rows = _mixed_rows(640, 300, 2, dmax, seed=11 + dmax)
    r = np.random.default_rng(5)
    rows += [sorted(r.choice(640, size=d, replace=False).tolist()) for d in [6] * 64 + [dmax] * 64]
    code = I.from_rows(640, rows)
    assert int(np.max(np.diff(code.row_ptr))) == dmax
    assert int(np.max(np.bincount(code.col_idx))) <= 14  # 128 + 15 Qm <= 2048 for every Qm below
    rng = np.random.default_rng(dmax)
    q0 = rng.integers(-20, 21, size=(131, 640)).astype(np.int8)
    for p in (dict(rule="offset", offset=1, msg_sat=127), dict(rule="normalized", norm_num=3, norm_shift=2, msg_sat=5),
              dict(rule="plain", msg_sat=3), dict(rule="normalized", norm_num=7, norm_shift=3, msg_sat=127)):
        for es in (0, 1):
            _int(L, code, q0, form, dict(p, max_iter=12, early_stop=es), kernel="pingpong")
