"""Frame error rates of the decoders on device-generated frames: random codewords
of the code (a pool made by the code's encoder, each frame with its own noise),
BPSK over AWGN from ldpc_awgn_llr_f32, quantized for the int8 decoders with
ldpc_quantize_llr.  A point runs until it has seen ``min_errors`` frame errors
or ``max_frames`` frames, and reports a Wilson 95 % interval.

  python -m paper_cs_0609090_gb300.fer [--workload qc_n7493] [--ebn0 2.0 2.5 3.0]
         [--min-errors 100] [--max-frames 1048576] [--out result.json]
         [--learned-beta beta.json]

compares offset min-sum (the workload's int8 decoder) in the flooding and the
layered schedule, plain min-sum, normalized min-sum in float32 and the
sum-product rule (the accuracy reference), all with early stop; with
--learned-beta also the learned-offset decoder (10 iterations) against the plain
int8 decoder at 10 and 30 iterations.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from . import ldpc
from .inputs import Encoder, make_workload


def wilson(errors: int, n: int, z: float = 1.96):
    p = errors / n
    den = 1 + z * z / n
    centre = (p + z * z / (2 * n)) / den
    half = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / den
    return [max(0.0, centre - half), centre + half]


class CodewordPool:
    """`n` random codewords of a code on the device: packed (bit v at byte v >> 3,
    bit v & 7, the layout of ldpc_awgn_llr_f32 and of the decoders' output) and
    unpacked."""

    def __init__(self, code_inputs, n: int, seed: int, device):
        cw = Encoder(code_inputs).random_codewords(n, seed=seed)
        self.n = n
        self.bits = torch.from_numpy(cw).to(device)
        self.packed = torch.from_numpy(np.packbits(cw, axis=1, bitorder="little")).to(device)

    def rows(self, start: int, F: int, device):
        idx = (torch.arange(F, device=device) + start) % self.n
        return self.packed[idx].contiguous(), self.bits[idx]


def run_point(decode_batch, n_vars: int, rate: float, ebn0_db: float, pool: CodewordPool, *, min_errors: int = 100,
              max_frames: int = 1 << 20, batch: int = 8192, seed: int = 99, device=None) -> dict:
    """FER of one decoder at one Eb/N0.  decode_batch(llr_f32 [F, N]) returns
    (decisions, iterations): decisions packed [F, ceil(N/8)] or unpacked [F, N]."""
    dev = device or pool.bits.device
    llr = torch.empty((batch, n_vars), dtype=torch.float32, device=dev)
    errors = done = iters_sum = 0
    while done < max_frames and errors < min_errors:
        F = min(batch, max_frames - done)
        packed, bits = pool.rows(done, F, dev)
        ldpc.ldpc_awgn_llr_f32(n_vars, seed, done, F, ebn0_db, ebn0_db, rate, packed, llr[:F])
        dec, iters = decode_batch(llr[:F])
        ref = packed if dec.shape[1] == packed.shape[1] else bits
        errors += int((dec != ref).any(dim=1).sum().item())
        iters_sum += int(iters.sum().item()) if torch.is_tensor(iters) else iters * F
        done += F
    return {"frames": done, "errors": errors, "fer": errors / done, "wilson95": wilson(errors, done),
            "mean_iters": iters_sum / done, "ebn0_db": ebn0_db}


def int8_decoder(code, params, delta: float, qc: int, batch: int, device):
    q = torch.empty((batch, code.n_vars), dtype=torch.int8, device=device)

    def run(llr):
        F = llr.shape[0]
        if params.dtype == ldpc.LDPC_DTYPE_INT8:
            ldpc.ldpc_quantize_llr(llr, F * code.n_vars, delta, qc, q[:F])
            bits, iters, _, _ = ldpc.decode(code, q[:F], params)
        else:
            bits, iters, _, _ = ldpc.decode(code, llr, params)
        return bits, iters
    return run


def learned_decoder(code, beta, K: int, batch: int, device):
    from .learned import LearnedDecoder
    dec = LearnedDecoder(code, K, batch, device)
    b = torch.as_tensor(beta, dtype=torch.float32, device=device).contiguous()

    def run(llr):
        z = dec.forward(llr, b)
        return (z <= 0).to(torch.uint8), K
    return run


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
    ap.add_argument("--ebn0", type=float, nargs="+", default=[2.0, 2.5, 3.0])
    ap.add_argument("--min-errors", type=int, default=100)
    ap.add_argument("--max-frames", type=int, default=1 << 20)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--pool", type=int, default=4096, help="random codewords in the transmitted pool")
    ap.add_argument("--learned-beta", default=None, help="JSON with 'beta' [K][classes]: adds the learned decoder")
    ap.add_argument("--only-learned", action="store_true", help="the learned comparison only")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    w = make_workload(args.workload, with_llr=False)
    code = ldpc.Code.from_inputs(w.code)
    dev = torch.device("cuda", code.device)
    rate = (w.code.n_vars - w.code.n_checks) / w.code.n_vars
    pool = CodewordPool(w.code, args.pool, seed=12345, device=dev)
    todo = {} if args.only_learned else {k: int8_decoder(code, v, w.delta, w.qc, args.batch, dev)
                                         for k, v in decoders(w).items()}
    if args.learned_beta:
        beta = np.asarray(json.load(open(args.learned_beta))["beta"], dtype=np.float32)
        todo[f"learned offsets float32, {beta.shape[0]} it"] = learned_decoder(code, beta, beta.shape[0],
                                                                               args.batch, dev)
        for it in (beta.shape[0], 30):
            p = ldpc.make_params(**dict(w.params, early_stop=1, max_iter=it))
            todo[f"plain int8 offset {w.params['offset']} LSB, {it} it"] = int8_decoder(code, p, w.delta, w.qc,
                                                                                     args.batch, dev)
    rows = []
    for name, run in todo.items():
        for eb in args.ebn0:
            r = dict(decoder=name, **run_point(run, w.code.n_vars, rate, eb, pool, min_errors=args.min_errors,
                                               max_frames=args.max_frames, batch=args.batch))
            rows.append(r)
            print(json.dumps(r), flush=True)
    if args.out:
        json.dump({"workload": args.workload, "codewords": f"random, pool of {args.pool} (encoder seed 12345)",
                   "stop": f">= {args.min_errors} frame errors or {args.max_frames} frames", "rows": rows},
                  open(args.out, "w"), indent=1)


if __name__ == "__main__":
    main()
