"""The 8-bit stored posterior (LDPC_POSTERIOR_SAT8: Z^(k)_n clamped to
[-127, 127] after every iteration, read clamped by the next one) against the
oracle's post_sat = 127, bit-exact: on the frame-resident packed kernel (the
N=7493 code) and the two-launch streaming kernel (N=7493 forced, and the
N=64800 code, sampled frames).  Also: the clamp changes results where the
posteriors pass 127, requests it does not cover are refused, and the
quasi-cyclic descriptor builds the same code with its block rows as layers."""
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


@pytest.mark.parametrize("early_stop", [1, 0])
@pytest.mark.parametrize("form", FORMS_INT)
def test_qc_7493_sat8(L, form, early_stop):
    w = I.make_workload("qc_n7493", n_frames=131, ebn0_db=2.5, frame_seed=3)
    p = dict(w.params, early_stop=early_stop, max_iter=20, posterior="sat8")
    h = L.Code.from_inputs(w.code)
    o = oracle_int(w.code, w.q0, form, p)
    for kern, want in (("auto", "onchip_half"), ("onchip_half", "onchip_half"), ("stream", "stream")):
        params = L.make_params(form=form, kernel=kern, **p)
        assert L.ldpc_kernel_choice(h.handle, params, 131) == want
        g = gpu_decode(h, w.code.n_vars, w.q0, params)
        assert_int_parity(g, o)
        assert np.abs(g["z"]).max() <= 127
    exact = oracle_int(w.code, w.q0, form, dict(p, posterior="exact"))
    assert np.abs(exact.z).max() > 127
    assert not np.array_equal(exact.z.clip(-127, 127), o.z)  # the clamp acts inside the iterations


@pytest.mark.parametrize("form", FORMS_INT)
def test_irr_64800_sat8_sampled(L, form):
    """The whole 1024-frame batch on the streaming kernel (what AUTO runs for
    the 8-bit posterior on a code too large for one SM); sampled frames."""
    w = I.make_workload("irr_n64800")
    p = dict(w.params, early_stop=1, posterior="sat8")
    h = L.Code.from_inputs(w.code)
    params = L.make_params(form=form, **p)
    assert L.ldpc_kernel_choice(h.handle, params, w.n_frames) == "stream"
    g = gpu_decode(h, w.code.n_vars, w.q0, params)
    frames = np.array([0, 1, 517, w.n_frames - 2, w.n_frames - 1])
    assert_int_parity({k: v[frames] for k, v in g.items()}, oracle_int(w.code, w.q0[frames], form, p))


def test_sat8_refusals(L):
    w = I.make_workload("qc_n7493", n_frames=2)
    h = L.Code.from_inputs(w.code)
    for kw in (dict(kernel="pingpong"), dict(kernel="onchip_int"), dict(kernel="persistent"),
               dict(kernel="cluster"), dict(form="two_scan"), dict(form="two_scan_1bit"),
               dict(schedule="layered"), dict(dtype="f32")):
        params = L.make_params(**dict(w.params, posterior="sat8", **kw))
        with pytest.raises(L.LdpcError) as e:
            L.ldpc_workspace_size(h.handle, params, 2)
        assert e.value.status == L.LDPC_ERR_UNSUPPORTED, kw
    with pytest.raises(L.LdpcError) as e:
        L.ldpc_workspace_size(h.handle, L.make_params(**dict(w.params, posterior=2)), 2)
    assert e.value.status == L.LDPC_ERR_INVALID_ARG


def test_qc_descriptor_code(L):
    """Code.from_qc (ldpc_code_create_qc) decodes like the CSR code, and its
    layers are the 24 block rows, on which the layered schedule matches the
    oracle's layered decoder."""
    w = I.make_workload("qc_n7493", n_frames=64, ebn0_db=2.5, frame_seed=4)
    S, Z = w.code.meta["shifts"], w.code.meta["Z"]
    hq = L.Code.from_qc(S, Z)
    info = L.ldpc_code_info(hq.handle)
    assert (info["n_vars"], info["n_checks"], info["n_edges"]) == (w.code.n_vars, w.code.n_checks, w.code.n_edges)
    n_layers, layer = L.ldpc_code_layers(hq.handle, w.code.n_checks)
    assert n_layers == S.shape[0] and np.array_equal(layer, np.arange(w.code.n_checks) // Z)
    p = dict(w.params, max_iter=15)
    for form in FORMS_INT:
        assert_int_parity(gpu_decode(hq, w.code.n_vars, w.q0, L.make_params(form=form, **p)),
                          oracle_int(w.code, w.q0, form, p))
    g = gpu_decode(hq, w.code.n_vars, w.q0, L.make_params(form="ss_1bit", schedule="layered", **p))
    o = oracle.decode_layered_int(w.code, w.q0.astype(np.int32), layer, rule=p["rule"], offset=p["offset"],
                                  msg_sat=p["msg_sat"], max_iter=p["max_iter"], early_stop=p["early_stop"])
    assert_int_parity(g, o)
