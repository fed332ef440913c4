"""Frame error rates of the decoders on device-generated frames: BPSK over AWGN
with the all-zero codeword (the decoders are symmetric), channel values from
ldpc_awgn_llr_f32, quantized for the int8 decoders with ldpc_quantize_llr.

  python -m paper_cs_0609090_gb300.fer [--workload qc_n7493] [--frames 65536]
         [--ebn0 2.0 2.5 3.0] [--out result.json]

compares offset min-sum (the workload's int8 decoder) in the flooding and the
layered schedule, plain min-sum, normalized min-sum in float32 and the
sum-product rule (the accuracy reference), all with early stop.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from . import ldpc
from .inputs import make_workload


def wilson(errors: int, n: int, z: float = 1.96):
    p = errors / n
    den = 1 + z * z / n
    centre = (p + z * z / (2 * n)) / den
    half = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / den
    return [max(0.0, centre - half), centre + half]


def fer(code: "ldpc.Code", params: "ldpc.ldpc_decode_params", n_frames: int, ebn0_db: float, *, rate: float,
        delta: float = 0.125, qc: int = 127, seed: int = 99, batch: int = 8192) -> dict:
    """FER and mean iterations of one decoder at one Eb/N0 (all-zero codeword)."""
    dev = torch.device("cuda", code.device)
    N = code.n_vars
    llr = torch.empty((batch, N), dtype=torch.float32, device=dev)
    q = torch.empty((batch, N), dtype=torch.int8, device=dev)
    errors = done = iters_sum = 0
    while done < n_frames:
        F = min(batch, n_frames - done)
        ldpc.ldpc_awgn_llr_f32(N, seed, done, F, ebn0_db, ebn0_db, rate, None, llr[:F])
        if params.dtype == ldpc.LDPC_DTYPE_INT8:
            ldpc.ldpc_quantize_llr(llr[:F], F * N, delta, qc, q[:F])
            bits, iters, _, _ = ldpc.decode(code, q[:F], params)
        else:
            bits, iters, _, _ = ldpc.decode(code, llr[:F], params)
        errors += int((bits != 0).any(dim=1).sum().item())
        iters_sum += int(iters.sum().item())
        done += F
    return {"frames": done, "errors": errors, "fer": errors / done, "wilson95": wilson(errors, done),
            "mean_iters": iters_sum / done, "ebn0_db": ebn0_db}


def decoders(w) -> dict:
    p = dict(w.params, early_stop=1)
    return {
        "min-sum offset int8 (flooding)": ldpc.make_params(**p),
        "min-sum offset int8 (layered)": ldpc.make_params(schedule="layered", **p),
        "min-sum plain int8": ldpc.make_params(**dict(p, rule="plain")),
        "normalized 0.75 float32": ldpc.make_params(dtype="f32", rule="normalized", norm_f32=0.75,
                                                    max_iter=p["max_iter"], early_stop=1),
        "sum-product float32": ldpc.make_params(dtype="f32", form="ss_fixed", rule="sum_product",
                                                max_iter=p["max_iter"], early_stop=1),
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="qc_n7493")
    ap.add_argument("--frames", type=int, default=1 << 16)
    ap.add_argument("--ebn0", type=float, nargs="+", default=[2.0, 2.5, 3.0])
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    w = make_workload(args.workload, with_llr=False)
    code = ldpc.Code.from_inputs(w.code)
    rate = (w.code.n_vars - w.code.n_checks) / w.code.n_vars
    rows = []
    for name, params in decoders(w).items():
        for eb in args.ebn0:
            r = dict(decoder=name, **fer(code, params, args.frames, eb, rate=rate, delta=w.delta, qc=w.qc))
            rows.append(r)
            print(json.dumps(r), flush=True)
    if args.out:
        json.dump({"workload": args.workload, "frames_per_point": args.frames, "rows": rows},
                  open(args.out, "w"), indent=1)


if __name__ == "__main__":
    main()
