"""Shared helpers for the GPU parity tests: run the CUDA path through the C ABI
and the CPU oracle on the same seeded inputs, and compare."""
import numpy as np

import oracle
from paper_cs_0609090_gb300 import inputs as I

FORMS_INT = ("ss_1bit", "ss_fixed")
KERNELS_INT = ("onchip_half", "onchip_int")


def gpu_decode(code_handle, n_vars, q0, params, want_llr=True):
    import torch
    from paper_cs_0609090_gb300 import ldpc
    t = torch.from_numpy(np.ascontiguousarray(q0)).cuda()
    bits, iters, ok, zo = ldpc.decode(code_handle, t, params, want_llr=want_llr)
    torch.cuda.synchronize()
    out = dict(bits=ldpc.unpack_bits(bits.cpu().numpy(), n_vars), iters=iters.cpu().numpy(),
               ok=ok.cpu().numpy())
    if want_llr:
        out["z"] = zo.cpu().numpy()
    return out


def oracle_int(code, q0, form, p):
    return oracle.decode_int(code, q0.astype(np.int32), form=form, rule=p.get("rule", "offset"),
                             offset=p.get("offset", 0), norm_num=p.get("norm_num", 3),
                             norm_shift=p.get("norm_shift", 2), msg_sat=p.get("msg_sat", 127),
                             max_iter=p["max_iter"], early_stop=p.get("early_stop", 1),
                             post_sat=127 if p.get("posterior", "exact") == "sat8" else 0)


def assert_int_parity(g, o):
    """Bit-exact equality of decisions, iteration counts, flags and posteriors."""
    for key in ("bits", "iters", "ok") + (("z",) if "z" in g else ()):
        a = np.asarray(g[key]).astype(np.int64)
        b = np.asarray(o[key]).astype(np.int64)
        if not np.array_equal(a, b):
            bad = np.nonzero(np.any((a != b).reshape(a.shape[0], -1), axis=1))[0]
            raise AssertionError(f"{key} differs on {bad.size} frames, first {bad[:8].tolist()}")
