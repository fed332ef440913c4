"""GPU vs oracle parity of the thread-block-cluster kernel (one frame pair over
the CTAs of a cluster) and of the multi-code persistent launch (several codes,
CTA sub-teams and clusters, work queue, CUDA graph replay, autotuning):
decisions, iteration counts, syndrome flags and final posteriors must be
bit-identical to the oracle's."""
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


def _cluster(L, code, q0, form, p):
    h = L.Code.from_inputs(code)
    g = gpu_decode(h, code.n_vars, q0, L.make_params(form=form, kernel="cluster", **p))
    assert_int_parity(g, oracle_int(code, q0, form, p))
    return g


@pytest.mark.parametrize("form", FORMS_INT)
@pytest.mark.parametrize("early_stop", [1, 0])
def test_cluster_kernel_small_codes(L, form, early_stop):
    """Codes that fit one CTA, forced onto a cluster (2 CTAs): the distributed
    shared-memory path against the oracle where the oracle is fast."""
    w = I.make_workload("reg36_n1008", n_frames=41, ebn0_db=1.8)
    _cluster(L, w.code, w.q0, form, dict(w.params, early_stop=early_stop))
    w = I.make_workload("qc_n7493", n_frames=13, ebn0_db=2.0)
    _cluster(L, w.code, w.q0, form, dict(w.params, early_stop=early_stop))


@pytest.mark.parametrize("form", FORMS_INT)
def test_cluster_kernel_edge_cases(L, form):
    w = I.make_workload("reg36_n1008", n_frames=9, ebn0_db=1.0)
    _cluster(L, w.code, w.q0[:1], form, w.params)                        # one frame: a ragged pair
    _cluster(L, w.code, w.q0, form, dict(w.params, max_iter=0))
    _cluster(L, w.code, w.q0, form, dict(w.params, max_iter=1, early_stop=0))
    g = _cluster(L, w.code, I.noiseless(w.codewords, 31), form, w.params)
    assert np.all(g["iters"] == 0) and np.all(g["ok"] == 1)
    rng = np.random.default_rng(5)
    q = rng.integers(-128, 128, size=(5, w.code.n_vars)).astype(np.int8)
    _cluster(L, w.code, q, form, dict(w.params, msg_sat=127, rule="plain", early_stop=0, max_iter=7))
    for rule in ("plain", "normalized"):
        _cluster(L, w.code, w.q0, form, dict(w.params, rule=rule, norm_num=5, norm_shift=3))


@pytest.mark.parametrize("form", FORMS_INT)
def test_cluster_kernel_staircase_16200(L, form):
    """A staircase code too large for one SM on a cluster (the library's own
    choice for it is the faster streaming kernel, which needs a workspace)."""
    c = I.staircase_code(16200, 32)
    w = I.make_workload("irr_n64800", n_frames=9, ebn0_db=1.5, code=c)
    p = dict(w.params, max_iter=30)
    h = L.Code.from_inputs(c)
    assert L.ldpc_workspace_size(h.handle, L.make_params(form=form, **p), 9) > 0
    assert L.ldpc_workspace_size(h.handle, L.make_params(form=form, kernel="cluster", **p), 9) == 0
    g = gpu_decode(h, c.n_vars, w.q0, L.make_params(form=form, kernel="cluster", **p))
    assert_int_parity(g, oracle_int(c, w.q0, form, p))


def _multi_oracle(ws, form):
    return [oracle_int(w.code, w.q0, form, w.params) for w in ws]


def _multi_check(L, mb, ws, ref):
    import torch
    torch.cuda.synchronize()
    for j, w in enumerate(ws):
        bits, iters, ok, zo = mb.outputs[j]
        g = dict(bits=L.unpack_bits(bits.cpu().numpy(), w.code.n_vars), iters=iters.cpu().numpy(),
                 ok=ok.cpu().numpy())
        if zo is not None:
            g["z"] = zo.cpu().numpy()
        try:
            assert_int_parity(g, ref[j])
        except AssertionError as e:
            raise AssertionError(f"job {j} ({w.name}): {e}")


def _batch(L, ws, form, tuning=None, want_llr=True):
    import torch
    codes = [L.Code.from_inputs(w.code) for w in ws]
    llrs = [torch.from_numpy(np.ascontiguousarray(w.q0)).cuda() for w in ws]
    params = [L.make_params(form=form, **w.params) for w in ws]
    return L.MultiBatch(codes, llrs, params, want_llr=want_llr, tuning=tuning), codes, llrs


SMALL_COUNTS = [7, 5, 9, 4, 6, 3, 3, 2]


@pytest.mark.parametrize("form", FORMS_INT)
@pytest.mark.parametrize("queue", [1, 2])
@pytest.mark.parametrize("large", [1, 2])
def test_multi_batch_eight_codes(L, form, queue, large):
    """All eight codes of the uneven batch (three do not fit one CTA: streaming
    decoder or clusters), ragged frame counts; dynamic queue and round-robin."""
    ws = I.make_multi_workload(frames=SMALL_COUNTS)
    mb, _, _ = _batch(L, ws, form, L.ldpc_multi_tuning(0, 0, 0, queue, large))
    info = mb.info()
    # per-edge messages of the N=7493 code (with its column table) exceed one CTA
    big = 1 if large == 2 else 2
    assert info["job_is_cluster"] == [0, 0, 0, 0, big * (form == "ss_fixed"), big, big, big]
    assert (info["cluster"] >= 2) == (large == 2)
    mb.decode()
    _multi_check(L, mb, ws, _multi_oracle(ws, form))


@pytest.mark.parametrize("form", FORMS_INT)
def test_multi_batch_local_only_and_subteams(L, form):
    """Codes that fit a CTA only (no cluster in the launch), several frame pairs
    per CTA on sub-teams, early stop on, mixed rules, a job without frames."""
    import dataclasses
    ws = I.make_multi_workload(frames=[61, 33, 17, 12, 0, 0, 0, 0], codes=[0, 1, 2, 3])
    for w in ws:
        w.params["max_iter"] = 25
    ws[1].params.update(rule="normalized", norm_num=3, norm_shift=2)
    empty = dataclasses.replace(ws[0], n_frames=0, q0=ws[0].q0[:0])
    for tt in (64, 128, 256):
        mb, _, _ = _batch(L, ws + [empty], form, L.ldpc_multi_tuning(1024, tt, 0, 1))
        info = mb.info()
        assert info["cluster"] == 1 and info["job_is_cluster"] == [0, 0, 0, 0, -1]
        assert info["job_pairs_per_cta"][0] == min(8, 1024 // tt)
        mb.decode()
        _multi_check(L, mb, ws, _multi_oracle(ws, form))


@pytest.mark.parametrize("overlap", [1, 2])
def test_multi_batch_cuda_graph_replay(L, overlap):
    """The launch is captured once in a CUDA graph and replayed on new channel
    values written into the same input buffers; the three codes on the
    streaming decoder in sequence (overlap 1) or forked onto side streams and
    joined back (overlap 2), checked directly and after the replays."""
    import torch
    form = "ss_1bit"
    ws = I.make_multi_workload(frames=[5, 4, 3, 6, 5, 2, 2, 1], frame_seed=7)
    mb, codes, llrs = _batch(L, ws, form, L.ldpc_multi_tuning(0, 0, 0, 0, 0, overlap))
    assert mb.info()["overlap"] == overlap
    mb.decode()
    _multi_check(L, mb, ws, _multi_oracle(ws, form))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        mb.decode(stream=s)           # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        mb.decode(stream=s)
    for seed in (8, 9):
        ws2 = I.make_multi_workload(frames=[5, 4, 3, 6, 5, 2, 2, 1], frame_seed=seed)
        for t, w in zip(llrs, ws2):
            t.copy_(torch.from_numpy(w.q0))
        for bits, iters, ok, zo in mb.outputs:
            bits.zero_(), iters.fill_(-1), ok.fill_(7)
        g.replay()
        _multi_check(L, mb, ws2, _multi_oracle(ws2, form))


@pytest.mark.parametrize("overlap", [0, 2])
def test_multi_batch_autotune(L, overlap):
    """The autotuner picks a shape (and, with overlap 0, the schedule of the
    streamed codes); a schedule fixed by the caller (2) is kept."""
    form = "ss_fixed"
    ws = I.make_multi_workload(frames=[8, 6, 4, 5, 7, 3, 2, 2], frame_seed=11)
    mb, _, _ = _batch(L, ws, form, L.ldpc_multi_tuning(0, 0, 0, 0, 0, overlap), want_llr=False)
    shape, ms = mb.autotune(reps=1)
    assert ms > 0 and shape.threads in (512, 1024) and shape.team_threads in (64, 128, 256)
    assert shape.large in (1, 2)
    if overlap:
        assert shape.overlap == overlap and mb.info()["overlap"] == overlap
    for bits, iters, ok, _ in mb.outputs:
        bits.zero_(), iters.fill_(-1), ok.fill_(7)
    mb.decode()
    _multi_check(L, mb, ws, _multi_oracle(ws, form))


@pytest.mark.parametrize("form", ["ss_1bit", "ss_fixed"])
@pytest.mark.parametrize("warps", [4, 16])
def test_multi_batch_stream_warps(L, form, warps):
    """The ping-pong row kernel of the streamed staircase codes at 4 and 16
    warps per CTA (16 and 64 checks per CTA) decodes exactly as the oracle;
    a value fixed by the caller survives the autotuner, 0 lets it choose (when
    its plan streams codes at all)."""
    ws = I.make_multi_workload(frames=[4, 3, 2, 5, 3, 9, 7, 5], frame_seed=12)
    mb, _, _ = _batch(L, ws, form, L.ldpc_multi_tuning(0, 0, 0, 0, 0, 2, warps))
    assert mb.info()["stream_warps"] == warps
    mb.decode()
    _multi_check(L, mb, ws, _multi_oracle(ws, form))
    shape, _ = mb.autotune(reps=1)
    assert shape.stream_warps == warps
    mb2, _, _ = _batch(L, ws, form, None)
    shape, _ = mb2.autotune(reps=1)
    # a plan that keeps every code inside the persistent launch (clusters) has
    # no ping-pong row kernel to tune
    streamed = 2 in mb2.info()["job_is_cluster"]
    assert shape.stream_warps in ((4, 8, 16) if streamed else (0,))
    mb2.decode()
    _multi_check(L, mb2, ws, _multi_oracle(ws, form))


def test_multi_rejects_bad_batches(L):
    import torch
    ws = I.make_multi_workload(frames=[3, 3, 0, 0, 0, 0, 0, 0], codes=[0, 1])
    codes = [L.Code.from_inputs(w.code) for w in ws]
    llrs = [torch.from_numpy(w.q0).cuda() for w in ws]
    with pytest.raises(L.LdpcError) as e:       # two forms in one batch
        L.MultiBatch(codes, llrs, [L.make_params(form="ss_1bit", **ws[0].params),
                                   L.make_params(form="ss_fixed", **ws[1].params)])
    assert e.value.status == L.LDPC_ERR_INVALID_ARG
    with pytest.raises(L.LdpcError) as e:       # float32 jobs are not batched
        L.MultiBatch(codes, llrs, [L.make_params(**dict(w.params, dtype="f32")) for w in ws])
    assert e.value.status == L.LDPC_ERR_UNSUPPORTED
    with pytest.raises(L.LdpcError) as e:       # more than 16 jobs
        L.MultiBatch(codes * 9, llrs * 9, [L.make_params(**ws[0].params)] * 18)
    assert e.value.status == L.LDPC_ERR_INVALID_ARG
    with pytest.raises(L.LdpcError) as e:       # a shape outside the documented ranges
        L.MultiBatch(codes, llrs, [L.make_params(**w.params) for w in ws], tuning=L.ldpc_multi_tuning(300, 0, 0, 0))
    assert e.value.status == L.LDPC_ERR_INVALID_ARG
    with pytest.raises(L.LdpcError) as e:       # stream_warps outside 0, 4, 8, 16
        L.MultiBatch(codes, llrs, [L.make_params(**w.params) for w in ws],
                     tuning=L.ldpc_multi_tuning(0, 0, 0, 0, 0, 0, 6))
    assert e.value.status == L.LDPC_ERR_INVALID_ARG
