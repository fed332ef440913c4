"""Learned offset min-sum: the offsets beta[k][c] of Section III's offset rule,
one per iteration k and check-degree class c, trained by gradient descent.

Every numerical step runs in the library's CUDA kernels (ldpc_learned_forward /
_loss / _backward, ldpc_adam_step, ldpc_awgn_llr_f32, ldpc_quantize_llr); this
module only allocates buffers with torch and sequences the calls.

  LearnedOffsetDecode.apply(llr, beta, decoder) -> Z^(K)   (torch.autograd.Function)
  train(...)                                                (C5 training loop)
  fer(...)                                                  frame error rates
"""
from __future__ import annotations

import json
import math
import time

import numpy as np
import torch

from . import ldpc


class LearnedDecoder:
    """Buffers for K learned iterations of one code on up to ``max_frames`` frames."""

    def __init__(self, code: "ldpc.Code", n_iters: int, max_frames: int, device=None):
        self.code = code
        self.K = int(n_iters)
        self.classes = ldpc.ldpc_code_degree_classes(code.handle)
        self.C = len(self.classes)
        self.max_frames = int(max_frames)
        self.device = torch.device("cuda", code.device) if device is None else device
        self.ws_bytes = ldpc.ldpc_learned_workspace_size(code.handle, self.K, self.max_frames)
        self._ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        self.frames = 0  # frames of the last forward
        # Number of forwards run so far: the workspace holds the checkpoints of
        # the latest one only, and a backward through an earlier one must not
        # read them.
        self.generation = 0

    def ws(self):
        base = (self._ws.data_ptr() + 255) & ~255

        class _P:
            def data_ptr(self):
                return base
        return _P()

    def ws_size(self, F: int) -> int:
        return ldpc.ldpc_learned_workspace_size(self.code.handle, self.K, F)

    def forward(self, llr: torch.Tensor, beta: torch.Tensor, want_z: bool = True):
        F, N = llr.shape
        assert F <= self.max_frames and N == self.code.n_vars and beta.shape == (self.K, self.C)
        z = torch.empty((F, N), dtype=torch.float32, device=llr.device) if want_z else None
        ldpc.ldpc_learned_forward(self.code.handle, self.K, beta, llr, F, z, self.ws(), self.ws_size(F))
        self.frames = F
        self.generation += 1
        return z

    def loss(self, target_bits=None, want_grad: bool = True) -> torch.Tensor:
        out = torch.empty(1, dtype=torch.float32, device=self.device)
        ldpc.ldpc_learned_loss(self.code.handle, self.K, self.frames, target_bits, out, want_grad, self.ws(),
                               self.ws_size(self.frames))
        return out

    def backward(self, beta: torch.Tensor, dz: torch.Tensor | None = None) -> torch.Tensor:
        db = torch.empty((self.K, self.C), dtype=torch.float32, device=self.device)
        ldpc.ldpc_learned_backward(self.code.handle, self.K, beta, dz, self.frames, db, self.ws(),
                                   self.ws_size(self.frames))
        return db


class LearnedOffsetDecode(torch.autograd.Function):
    """Z^(K) = decode(llr; beta) with the hand-written adjoint as its backward.
    Gradients flow to ``beta`` only (the channel values are data).

    The adjoint reads the per-iteration checkpoints that the forward left in the
    decoder's workspace, and a decoder keeps those of its latest forward only.
    So the backward of an apply must run before the next apply on the same
    decoder (or use one decoder per apply); otherwise it raises instead of
    returning the gradient of the wrong frames."""

    @staticmethod
    def forward(ctx, llr, beta, decoder: LearnedDecoder):
        llr = llr.contiguous().float()
        beta_c = beta.detach().contiguous().float()
        z = decoder.forward(llr, beta_c)
        ctx.decoder = decoder
        ctx.generation = decoder.generation
        ctx.save_for_backward(beta_c)
        return z

    @staticmethod
    def backward(ctx, grad_z):
        (beta_c,) = ctx.saved_tensors
        if ctx.decoder.generation != ctx.generation:
            raise RuntimeError(
                f"LearnedOffsetDecode.backward: the decoder ran {ctx.decoder.generation - ctx.generation} "
                "forward(s) after this one, so its workspace no longer holds this forward's checkpoints; "
                "run backward before the next apply or use a separate LearnedDecoder per apply")
        db = ctx.decoder.backward(beta_c, grad_z.contiguous().float())
        return None, db, None


def initial_beta(K: int, C: int, value: float = 0.25) -> np.ndarray:
    return np.full((K, C), value, dtype=np.float32)


def train(code, K: int = 10, total_frames: int = 1 << 20, batch: int = 8192, ebn0=(1.5, 3.5), lr: float = 0.01,
          seed: int = 1234, beta0: float = 0.25, log=None) -> dict:
    """Trains beta on all-zero codewords over BPSK/AWGN with per-frame Eb/N0
    uniform in ``ebn0`` (frames generated on the device), mean BCE of sigma(-Z^(K))
    as the loss, Adam.  Returns the learned table and the loss trace."""
    dev = torch.device("cuda", code.device)
    dec = LearnedDecoder(code, K, batch, dev)
    rate = (code.n_vars - code.n_checks) / code.n_vars
    beta = torch.from_numpy(initial_beta(K, dec.C, beta0)).to(dev)
    m = torch.zeros_like(beta)
    v = torch.zeros_like(beta)
    llr = torch.empty((batch, code.n_vars), dtype=torch.float32, device=dev)
    losses = []
    steps = max(1, total_frames // batch)
    t0 = time.time()
    for step in range(1, steps + 1):
        ldpc.ldpc_awgn_llr_f32(code.n_vars, seed, (step - 1) * batch, batch, ebn0[0], ebn0[1], rate, None, llr)
        dec.forward(llr, beta, want_z=False)
        loss = dec.loss(None, want_grad=True)
        grad = dec.backward(beta, None)
        ldpc.ldpc_adam_step(beta, grad, m, v, beta.numel(), step, lr)
        if step % 8 == 0 or step == steps:
            losses.append((step, float(loss.item())))
            if log:
                log(f"step {step}/{steps} loss {losses[-1][1]:.5f} beta[0] {beta[0].tolist()}")
    torch.cuda.synchronize()
    return {"beta": beta.cpu().numpy(), "losses": losses, "steps": steps, "batch": batch,
            "train_seconds": time.time() - t0, "classes": dec.classes}


def fer(code, n_frames: int, ebn0_db: float, *, learned_beta=None, K: int = 10, int_params=None, delta=0.125,
        qc=127, seed=99, batch: int = 8192) -> dict:
    """Frame error rate on all-zero codewords at ``ebn0_db``: the learned float32
    decoder (learned_beta given, K iterations, decision on Z^(K)) or the plain int8
    decoder (int_params: ldpc_decode_params fields).  A frame is in error when any
    decision differs from the transmitted bit."""
    dev = torch.device("cuda", code.device)
    rate = (code.n_vars - code.n_checks) / code.n_vars
    N = code.n_vars
    llr = torch.empty((batch, N), dtype=torch.float32, device=dev)
    errors = 0
    done = 0
    iters_sum = 0
    dec = None
    if learned_beta is not None:
        dec = LearnedDecoder(code, K, batch, dev)
        beta = torch.as_tensor(learned_beta, dtype=torch.float32, device=dev).contiguous()
    else:
        q = torch.empty((batch, N), dtype=torch.int8, device=dev)
        params = ldpc.make_params(**int_params)
    while done < n_frames:
        F = min(batch, n_frames - done)
        ldpc.ldpc_awgn_llr_f32(N, seed, done, F, ebn0_db, ebn0_db, rate, None, llr[:F])
        if dec is not None:
            z = dec.forward(llr[:F], beta)
            errors += int((z <= 0).any(dim=1).sum().item())
            iters_sum += K * F
        else:
            ldpc.ldpc_quantize_llr(llr[:F], F * N, delta, qc, q[:F])
            bits, iters, ok, _ = ldpc.decode(code, q[:F], params)
            errors += int((bits != 0).any(dim=1).sum().item())
            iters_sum += int(iters.sum().item())
        done += F
    p = errors / done
    z = 1.96
    den = 1 + z * z / done
    centre = (p + z * z / (2 * done)) / den
    half = z * math.sqrt(p * (1 - p) / done + z * z / (4 * done * done)) / den
    return {"frames": done, "errors": errors, "fer": p, "wilson95": [max(0.0, centre - half), centre + half],
            "mean_iters": iters_sum / done, "ebn0_db": ebn0_db}


def main():
    import argparse
    from .inputs import make_workload
    ap = argparse.ArgumentParser(description="train learned offsets on the N=7493 QC code and compare FER")
    ap.add_argument("--frames", type=int, default=1 << 20)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--fer-frames", type=int, default=1 << 16)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    w = make_workload("qc_n7493", with_llr=False)
    code = ldpc.Code.from_inputs(w.code)
    res = train(code, total_frames=args.frames, batch=args.batch, log=print)
    report = {"train": {k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in res.items()}, "fer": []}
    plain = dict(w.params)
    for eb in (2.0, 2.5, 3.0):
        row = {"ebn0_db": eb,
               "learned_f32_10it": fer(code, args.fer_frames, eb, learned_beta=res["beta"], K=10),
               "plain_int8_10it": fer(code, args.fer_frames, eb, int_params=dict(plain, max_iter=10)),
               "plain_int8_30it": fer(code, args.fer_frames, eb, int_params=dict(plain, max_iter=30))}
        report["fer"].append(row)
        print(json.dumps(row))
    if args.out:
        json.dump(report, open(args.out, "w"), indent=1)


if __name__ == "__main__":
    main()
