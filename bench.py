#!/usr/bin/env python3
"""Decoded-information throughput of the single-scan min-sum decoder on GB300.

One step = one ldpc_decode_batch call over the whole workload batch with early
stop off (every frame runs the fixed iteration count), LLRs already resident
in HBM.  ``value`` = decoded information bits (F * K per step) per second,
whole job over all ranks; ``e2e`` is the same through the C ABI with the LLRs
copied from pinned host memory and the decisions/iterations/flags copied back
inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload irr_n64800]
                  [--form ss_1bit|ss_fixed|two_scan|two_scan_1bit] [--impl ours|reference]

The default workload is the largest single-GPU configuration: the N=64800 rate
1/2 staircase code, 1024 frames, 50 iterations, int8, Section V form.  The same
run times the comparison forms on the same frames (the per-edge single scan and
the two-scan with per-edge or Section V message storage) and reports them under
``comparisons``, with the single-scan/two-scan time ratios; it also measures the
frame error rate at the workload's Eb/N0 with early stop on (``fer``).

``--workload multi8`` times the uneven eight-code batch (ldpc_multi_* plan,
autotuned, one CUDA graph replay per step); ``--workload learned_qc_n7493`` one
training step of the learned offset decoder (8192 device-generated frames).

``--impl reference`` times the CPU oracle (the only reference this method has)
on a bounded sample of the same workload and prints the same JSON line.
Multi-GPU (torchrun): every rank decodes its own batch (frames are independent;
weak scaling, no collective on the data path); time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_cs_0609090_gb300 import inputs as I  # noqa: E402

METRIC = "decoded info Gbit/s at fixed iters, single-scan vs two-scan; FER @ stated Eb/N0"
UNIT = "Gbit/s"


def algorithmic_bytes(code, form: str, iters: int, frames: int, dtype: str = "int8") -> dict:
    """Streaming-model bytes of one decode: per frame-iteration 2 b_z N + 2 S_L
    (read and write of the posterior and of the message state) plus per frame
    the LLRs in, packed decisions out and 5 bytes of iteration count/flag.
    int8: b_z = 2, S_L = (ceil(d_c/8) + 3) M (Section V) or E (per edge);
    float32: b_z = 4, S_L = (ceil(d_c/8) + 9) M or 4 E."""
    N, M, E = code.n_vars, code.n_checks, code.n_edges
    dmax = int(code.row_degrees().max())
    f32 = dtype == "f32"
    b_z = 4 if f32 else 2
    if form == "ss_1bit":
        s_l = ((dmax + 7) // 8 + (9 if f32 else 3)) * M
    elif form == "ss_fixed":
        s_l = (4 if f32 else 1) * E
    else:  # two-scan: Z_mn and L_mn cells read and written, plus q0 and decisions
        s_l = None
    if form == "two_scan_1bit":
        # two-scan with the Section V message storage: Z_mn read and written per
        # edge, the state written and read once, q0 and decisions
        b_it = 2 * E + 2 * ((dmax + 7) // 8 + 3) * M + N + N // 8
    elif s_l is None:
        b_it = (4 if not f32 else 16) * E + N + N // 8
    else:
        b_it = 2 * b_z * N + 2 * s_l
    b_io = N * (4 if f32 else 1) + (N + 7) // 8 + 5
    return dict(per_frame_iter=b_it, per_frame_io=b_io, per_launch=frames * (iters * b_it + b_io))


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, max, throttle reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


KERNEL_SOURCES = {"onchip_h2_kernel": "onchip_h2.cu", "onchip_int8_kernel": "onchip_int8.cu", "pp_kernel": "persist.cu", "pp2_rows": "pingpong.cu",
                  "ts_horizontal": "twoscan_stream.cu",
                  "onchip_twoscan_kernel": "onchip_twoscan.cu", "h2s_rows": "stream.cu", "f32s_rows": "stream_f32.cu",
                  "layered_kernel": "layered_h2.cu"}


def code_text(src: str) -> str:
    """C/C++/CUDA source without its comments and with whitespace runs collapsed:
    what the compiler sees, so that editing a comment keeps the hash."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c == '"' or c == "'":  # literal: copy through its closing quote
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash(kernel: str) -> str:
    """Hash of the code (comments left out) of the translation unit that defines
    ``kernel`` and of every local header it includes (transitively): the sources
    its machine code comes from."""
    csrc = os.path.join(ROOT, "paper_cs_0609090_gb300", "csrc")
    seen, todo = [], [os.path.join(csrc, KERNEL_SOURCES[kernel])]
    while todo:
        f = os.path.normpath(todo.pop(0))
        if f in seen:
            continue
        seen.append(f)
        for inc in re.findall(r'^#include "([^"]+)"', open(f).read(), flags=re.M):
            todo.append(os.path.join(os.path.dirname(f), inc))
    h = hashlib.sha256()
    for f in sorted(seen, key=lambda x: os.path.relpath(x, ROOT)):
        h.update(os.path.relpath(f, ROOT).encode())
        h.update(code_text(open(f, encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


def profiled(kernel: str, workload: str, form: str, key: str = "dram_bytes_per_launch"):
    """A per-launch figure from the committed ncu summaries (DRAM bytes, or
    executed warp instructions), if it was taken on the current sources of that
    kernel; otherwise None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p) or kernel not in KERNEL_SOURCES:
        return None
    d = json.load(open(p))
    e = d.get(f"{kernel}/{workload}/{form}")
    if not e or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    return e.get(key)


def profiled_traffic(kernel: str, workload: str, form: str):
    return profiled(kernel, workload, form, "dram_bytes_per_launch")


# Kernels that keep the frame state on chip: HBM carries only the LLRs and the
# results, so their bound is instruction issue, reported against the issue peak
# (every SM has 4 schedulers, each issuing at most one warp instruction per
# clock); the streaming-model HBM fraction is reported beside it.
ON_CHIP_KERNELS = ("onchip_h2_kernel", "onchip_int8_kernel", "onchip_twoscan_kernel")
SCHEDULERS_PER_SM = 4


def roofline_line(kname, w, form, dtype, F, ms_step, clocks, sm_count):
    ab = algorithmic_bytes(w.code, form, w.params["max_iter"], F, dtype)
    peaks = measured_peaks()
    achieved = ab["per_launch"] / (ms_step * 1e-3) / 1e9
    hbm = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": achieved / peaks["hbm_gbs"], "traffic": profiled_traffic(kname, w.name, form),
           "peak_source": peaks["source"] + " copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
           "algorithmic_bytes_per_launch": ab["per_launch"], "bytes_per_frame_iter": ab["per_frame_iter"],
           "kernel": kname, "kernel_ms": ms_step}
    inst = profiled(kname, w.name, form, "warp_inst_per_launch")
    mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz")
    if inst is None or not mhz:
        return hbm
    peak = sm_count * SCHEDULERS_PER_SM * mhz * 1e6 / 1e9
    got = inst / (ms_step * 1e-3) / 1e9
    if kname not in ON_CHIP_KERNELS:
        # streaming kernels: HBM is the reported bound; the issue rate they reach
        # shows how close the instruction count brings them to the other limit
        hbm["issue_effective"] = {"achieved": got, "peak": peak, "unit": "G warp-inst/s", "frac": got / peak,
                                  "warp_inst_per_launch": inst}
        return hbm
    return {"bound": "alu", "achieved": got, "peak": peak, "unit": "G warp-inst/s", "frac": got / peak,
            "traffic": hbm["traffic"],
            "peak_source": f"instruction issue: {sm_count} SMs x {SCHEDULERS_PER_SM} schedulers x 1 warp "
                           f"instruction per clock x {mhz:.0f} MHz (SM clock sampled during the timed steps)",
            "warp_inst_per_launch": inst, "inst_source": "ncu smsp__inst_executed.sum, profiles/traffic.json",
            "kernel": kname, "kernel_ms": ms_step,
            "hbm_effective": {k: hbm[k] for k in ("achieved", "peak", "unit", "frac", "peak_source",
                                                 "algorithmic_bytes_per_launch", "bytes_per_frame_iter")}}


def kernel_name(form: str, dtype: str, schedule: str, chosen: str, ws_bytes: int, code) -> str:
    """The kernel that dominates a decode of this request (the one the roofline
    line describes)."""
    if schedule == "layered":
        return "layered_kernel"
    if form in ("two_scan", "two_scan_1bit"):
        return "ts_horizontal" if ws_bytes > 0 else "onchip_twoscan_kernel"
    named = {"onchip_int": "onchip_int8_kernel", "onchip_half": "onchip_h2_kernel", "cluster": "multi_h2_kernel",
             "persistent": "pp_kernel", "pingpong": "pp2_rows"}
    if chosen in named:
        return named[chosen]
    if chosen == "stream":
        return "f32s_rows" if dtype == "f32" else "h2s_rows"
    return "onchip_h2_kernel"


def cpu_oracle_sample(w, form: str, budget_s: float, max_frames: int, layers=None):
    """Times the CPU oracle on successive chunks of the workload's frames until
    ``budget_s`` seconds of wall time or ``max_frames`` frames (the layered
    oracle when ``layers`` is given)."""
    import oracle
    p = w.params
    chunk = max(oracle.default_threads() * 2, 8)
    done, t_total = 0, 0.0
    kw = dict(rule=p["rule"], offset=p.get("offset", 0), norm_num=p.get("norm_num", 3),
              norm_shift=p.get("norm_shift", 2), msg_sat=p["msg_sat"], max_iter=p["max_iter"],
              early_stop=p.get("early_stop", 0))
    while done < max_frames and t_total < budget_s:
        q = w.q0[done % w.n_frames:][:chunk]
        t0 = time.perf_counter()
        if layers is not None:
            oracle.decode_layered_int(w.code, q, layers, **kw)
        else:
            # the two-scan with the Section V storage computes the two-scan's integers
            oracle.decode_int(w.code, q, form="two_scan" if form == "two_scan_1bit" else form, **kw)
        t_total += time.perf_counter() - t0
        done += q.shape[0]
    gbps = done * w.K / t_total / 1e9
    return dict(value=gbps, unit=UNIT, cores=oracle.default_threads(), kind="oracle",
                sample=f"{done} of {w.n_frames} frames of {w.name}, {p['max_iter']} iterations, "
                       f"early stop {'on' if p.get('early_stop', 0) else 'off'}, {form}, {t_total:.1f} s"), t_total / done


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    if args.workload == "learned_qc_n7493":
        wl = I.make_workload("qc_n7493", n_frames=64, ebn0_db=2.5, zero_codeword=True)
        budget = float(os.environ.get("BENCH_REF_BUDGET_S", "4"))
        vals = []
        for s in range(args.warmup + args.steps):
            info = cpu_oracle_learned_sample(wl, 10, budget if s >= args.warmup else 1.0)
            if s >= args.warmup:
                vals.append(info["value"])
        val = float(np.median(vals))
        info["value"] = val
        line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 8192 * wl.K / (val * 1e9) * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "learned_qc_n7493", "frames_per_step": 8192, "iters": 10},
                "impl": "reference", "cpu_baseline": info,
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    if args.workload == "multi8":
        ws = I.make_multi_workload()
        for w in ws:
            w.params["early_stop"] = 0
        budget = float(os.environ.get("BENCH_REF_BUDGET_S", "4"))
        vals = []
        for s in range(args.warmup + args.steps):
            info = cpu_oracle_multi_sample(ws, args.form, budget if s >= args.warmup else 1.0)
            if s >= args.warmup:
                vals.append(info["value"])
        val = float(np.median(vals))
        info["value"] = val
        bits = sum(w.n_frames * w.K for w in ws)
        line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": bits / (val * 1e9) * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
                "config": {"workload": "multi8", "form": args.form, "codes": [w.name for w in ws],
                           "n_frames": [w.n_frames for w in ws], "iters": 30},
                "impl": "reference", "cpu_baseline": info,
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    w = I.make_workload(args.workload)
    w.params["early_stop"] = 0
    budget = float(os.environ.get("BENCH_REF_BUDGET_S", "4"))
    per_step, step_ms = [], []
    info = None
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        info, sec_per_frame = cpu_oracle_sample(w, args.form, budget_s=budget if s >= args.warmup else 1.0,
                                                max_frames=w.n_frames)
        if s >= args.warmup:
            per_step.append(info["value"])
            step_ms.append((time.perf_counter() - t0) * 1e3)
    val = float(np.median(per_step))
    info["value"] = val
    # each step decodes a bounded sample of the batch: ms_per_step is that
    # sample's wall time, value its throughput; a whole-batch step would take
    # full_batch_ms_estimate (the same throughput over all frames)
    ms = float(np.median(step_ms))
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int8", "data": "synthetic",
            "config": {"workload": w.name, "form": args.form, "n_frames": w.n_frames,
                       "iters": w.params["max_iter"], "N": w.code.n_vars, "K": w.K,
                       "step": "a bounded sample of the batch per step (cpu_baseline.sample)",
                       "full_batch_ms_estimate": w.n_frames * w.K / (val * 1e9) * 1e3},
            "impl": "reference", "cpu_baseline": info,
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_oracle_multi_sample(ws, form: str, budget_s: float):
    """Times the CPU oracle on frames of every code of the batch in turn (the
    same frames per code share) until ``budget_s`` seconds."""
    import oracle
    chunk = max(oracle.default_threads(), 4)
    t_total, bits_done, frames_done = 0.0, 0, 0
    rnd = 0
    while t_total < budget_s:
        for w in ws:
            p = w.params
            q = w.q0[(rnd * chunk) % w.n_frames:][:chunk]
            t0 = time.perf_counter()
            oracle.decode_int(w.code, q, form=form, rule=p["rule"], offset=p.get("offset", 0),
                              norm_num=p.get("norm_num", 3), norm_shift=p.get("norm_shift", 2),
                              msg_sat=p["msg_sat"], max_iter=p["max_iter"], early_stop=0)
            t_total += time.perf_counter() - t0
            bits_done += q.shape[0] * w.K
            frames_done += q.shape[0]
        rnd += 1
    return dict(value=bits_done / t_total / 1e9, unit=UNIT, cores=oracle.default_threads(), kind="oracle",
                sample=f"{frames_done} frames, {chunk} per code per round over the 8 codes of multi8, "
                       f"30 iterations, early stop off, {form}, {t_total:.1f} s")


def multi_overlap_ab(ldpc, codes, llrs, params, shape, flush, stream, reps=25, warm=5):
    """The autotuned shape with the streamed codes in sequence (overlap 1) and
    overlapped on side streams (overlap 2): median ms of graph replays, each
    after a 256 MB L2 flush."""
    import torch
    out = {}
    for ov, name in ((1, "sequential"), (2, "overlapped")):
        t = ldpc.ldpc_multi_tuning(**dict({f: getattr(shape, f) for f, _ in shape._fields_}, overlap=ov))
        with torch.cuda.stream(stream):
            mb = ldpc.MultiBatch(codes, llrs, params, tuning=t)
            for _ in range(3):
                mb.decode(stream=stream)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            mb.decode(stream=stream)
        evs = []
        with torch.cuda.stream(stream):
            for s in range(warm + reps):
                flush.fill_(s & 0xff)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                g.replay()
                b.record(stream)
                evs.append((a, b))
        torch.cuda.synchronize()
        out[name + "_ms"] = float(np.median([a.elapsed_time(b) for a, b in evs[warm:]]))
        del g, mb
    out["note"] = "autotuned shape, overlap fixed each way; median of graph replays, L2 flushed before each"
    return out


def run_multi(args, world, rank, local):
    """The uneven eight-code batch: one plan (ldpc_multi_*), autotuned, captured
    once in a CUDA graph; a step is one graph replay decoding every frame of
    every code."""
    import torch
    from paper_cs_0609090_gb300 import ldpc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ws = I.make_multi_workload(frame_seed=1 + rank)
    for w in ws:
        w.params["early_stop"] = 0
    codes = [ldpc.Code.from_inputs(w.code, device=local) for w in ws]
    llrs = [torch.from_numpy(w.q0).to(dev) for w in ws]
    params = [ldpc.make_params(form=args.form, **w.params) for w in ws]
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        mb = ldpc.MultiBatch(codes, llrs, params)
        shape, tuned_ms = mb.autotune(reps=2, stream=stream)
    info = mb.info()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            mb.decode(stream=stream)
    torch.cuda.synchronize()
    for (bits, iters, ok, _), w in zip(mb.outputs, ws):
        assert int(iters.min()) == w.params["max_iter"] and int(iters.max()) == w.params["max_iter"]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        mb.decode(stream=stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.fill_(s & 0xff)
            evs[s][0].record(stream)
            graph.replay()
            evs[s][1].record(stream)
    torch.cuda.synchronize()
    total_ms = float(np.sum([a.elapsed_time(b) for a, b in evs]))

    h_llrs = [torch.from_numpy(w.q0).pin_memory() for w in ws]
    h_out = [tuple(t.cpu().pin_memory() for t in o[:3]) for o in mb.outputs]
    e2e_evs = []
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.fill_(s & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for d, h in zip(llrs, h_llrs):
                d.copy_(h, non_blocking=True)
            mb.decode(stream=stream)
            for o, h in zip(mb.outputs, h_out):
                for dt, ht in zip(o[:3], h):
                    ht.copy_(dt, non_blocking=True)
            b.record(stream)
            e2e_evs.append((a, b))
    torch.cuda.synchronize()
    clocks = sampler.stop()
    e2e_ms = float(np.sum([a.elapsed_time(b) for a, b in e2e_evs]))
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms, e2e_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms, e2e_ms = float(t[0]), float(t[1])
        dist.barrier()
    if rank != 0:
        return 0
    ms_step = total_ms / args.steps
    info_bits = sum(w.n_frames * w.K for w in ws)
    value = world * info_bits / (ms_step * 1e-3) / 1e9
    e2e_val = world * info_bits / (e2e_ms / args.steps * 1e-3) / 1e9
    ab = sum(algorithmic_bytes(w.code, args.form, w.params["max_iter"], w.n_frames)["per_launch"] for w in ws)
    peaks = measured_peaks()
    achieved = ab / (ms_step * 1e-3) / 1e9
    # streamed codes: the ping-pong decoder (checks of degree <= 8: init + one row
    # pass per iteration + final syndrome + output) or the two-launch decoder
    streamed = [w for w, v in zip(ws, info["job_is_cluster"]) if v == 2]
    launches = (1 if len(streamed) < len(ws) else 0) + sum(
        3 + (1 if int(np.diff(w.code.row_ptr).max()) <= 8 else 2) * 30 for w in streamed)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int8", "data": "synthetic",
            "config": {"workload": "multi8", "form": args.form, "codes": [w.name for w in ws],
                       "n_frames": [w.n_frames for w in ws], "iters": 30, "early_stop": 0,
                       "ebn0_db": [w.ebn0_db for w in ws], "graph": "one CUDA graph replay per step",
                       "l2": "flushed between timed steps (256 MB write)",
                       "plan": {k: info[k] for k in ("threads", "team_threads", "cluster", "queue", "large",
                                                    "overlap", "stream_warps", "grid", "smem_bytes",
                                                    "job_is_cluster", "job_pairs_per_cta")},
                       "autotune_ms": tuned_ms},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(sum(w.q0.nbytes for w in ws)),
                    "d2h_bytes_per_step": int(sum(sum(t.numel() * t.element_size() for t in o[:3])
                                                  for o in mb.outputs))},
            "gpu_launches": args.steps * launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                         "peak_source": peaks["source"] + " copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                         "algorithmic_bytes_per_launch": ab,
                         "kernel": "graph (multi_h2_kernel + streaming kernels of the codes that do not fit a CTA)",
                         "kernel_ms": ms_step},
            "clocks": clocks}
    if not args.no_compare and world == 1:
        line["overlap_ab"] = multi_overlap_ab(ldpc, codes, llrs, params, shape, flush, stream)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_multi_sample(ws, args.form,
                                                       float(os.environ.get("BENCH_CPU_BUDGET_S", "12")))
    print(json.dumps(line), flush=True)
    return 0


def learned_step_bytes(code, K: int, F: int) -> int:
    """Algorithmic bytes of one training step (float32 Section V decoder, K
    iterations): per frame-iteration the forward reads Z^(k-1) and the state and
    writes both as checkpoints (2*4N + 2*S_L); the adjoint reads Z^(k-1), both
    states and dZ^(k) and writes dZ^(k-1) (12N + 2*S_L); S_L = (ceil(d_c/8)+9) M."""
    N, M = code.n_vars, code.n_checks
    s_l = ((int(code.row_degrees().max()) + 7) // 8 + 9) * M
    return F * K * (20 * N + 4 * s_l) + F * N * 4


def cpu_oracle_learned_sample(w, K: int, budget_s: float):
    """Times the oracle's FP64 forward + reverse-mode gradient on frames of the batch."""
    import oracle
    tab = np.full((K, w.code.n_checks), 0.25)
    chunk = max(oracle.default_threads(), 4)
    done, t_total = 0, 0.0
    while t_total < budget_s:
        q = w.llr[done % w.n_frames:][:chunk]
        t0 = time.perf_counter()
        oracle.learned_grad(w.code, q, tab)
        t_total += time.perf_counter() - t0
        done += q.shape[0]
    return dict(value=done * w.K / t_total / 1e9, unit=UNIT, cores=oracle.default_threads(), kind="oracle",
                sample=f"{done} frames of {w.name}, FP64 forward + reverse-mode gradient over {K} iterations, "
                       f"{t_total:.1f} s")


def run_learned(args, world, rank, local):
    """One training step of the learned offset decoder on the N=7493 QC code:
    device AWGN frames (Eb/N0 ~ U[1.5, 3.5] dB, all-zero codeword), float32
    forward over 10 iterations with checkpoints, BCE, hand-written adjoint, Adam."""
    import torch
    from paper_cs_0609090_gb300 import ldpc, learned
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    K, B = 10, (args.frames or 8192)
    w = I.make_workload("qc_n7493", n_frames=B, with_llr=False)
    code = ldpc.Code.from_inputs(w.code, device=local)
    dec = learned.LearnedDecoder(code, K, B, dev)
    rate = (w.code.n_vars - w.code.n_checks) / w.code.n_vars
    beta = torch.from_numpy(learned.initial_beta(K, dec.C)).to(dev)
    m, v = torch.zeros_like(beta), torch.zeros_like(beta)
    llr = torch.empty((B, w.code.n_vars), dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    counter = [0]

    def step(gen=True):
        counter[0] += 1
        if gen:
            ldpc.ldpc_awgn_llr_f32(w.code.n_vars, 1234 + rank, counter[0] * B, B, 1.5, 3.5, rate, None, llr,
                                   stream=stream)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ldpc.ldpc_learned_forward(code.handle, K, beta, llr, B, None, dec.ws(), dec.ws_size(B), stream)
        ev[0].record(stream)
        loss = torch.empty(1, dtype=torch.float32, device=dev)
        ldpc.ldpc_learned_loss(code.handle, K, B, None, loss, True, dec.ws(), dec.ws_size(B), stream)
        ev[1].record(stream)
        grad = torch.empty_like(beta)
        ldpc.ldpc_learned_backward(code.handle, K, beta, None, B, grad, dec.ws(), dec.ws_size(B), stream)
        ev[2].record(stream)
        ldpc.ldpc_adam_step(beta, grad, m, v, beta.numel(), counter[0], 0.01, stream=stream)
        ev[3].record(stream)
        return loss, ev

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    rec = []
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.fill_(s & 0xff)
            ldpc.ldpc_awgn_llr_f32(w.code.n_vars, 1234 + rank, (1000 + s) * B, B, 1.5, 3.5, rate, None, llr,
                                   stream=stream)
            a = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, ev = step(gen=False)
            rec.append((a, ev))
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(ev[3]) for a, ev in rec]
    phases = {"forward_ms": float(np.mean([a.elapsed_time(ev[0]) for a, ev in rec])),
              "loss_ms": float(np.mean([ev[0].elapsed_time(ev[1]) for _, ev in rec])),
              "backward_ms": float(np.mean([ev[1].elapsed_time(ev[2]) for _, ev in rec])),
              "adam_ms": float(np.mean([ev[2].elapsed_time(ev[3]) for _, ev in rec]))}
    total_ms = float(np.sum(step_ms))
    # end to end: the batch's channel values from pinned host memory, the loss back
    h_llr = torch.empty((B, w.code.n_vars), dtype=torch.float32).pin_memory()
    h_llr.copy_(llr.cpu())
    h_loss = torch.empty(1, dtype=torch.float32).pin_memory()
    e2e = []
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.fill_(s & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            llr.copy_(h_llr, non_blocking=True)
            loss, _ = step(gen=False)
            h_loss.copy_(loss, non_blocking=True)
            b.record(stream)
            e2e.append((a, b))
    torch.cuda.synchronize()
    clocks = sampler.stop()
    e2e_ms = float(np.sum([a.elapsed_time(b) for a, b in e2e]))
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms, e2e_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms, e2e_ms = float(t[0]), float(t[1])
        dist.barrier()
    if rank != 0:
        return 0
    ms_step = total_ms / args.steps
    value = world * B * w.K / (ms_step * 1e-3) / 1e9
    ab = learned_step_bytes(w.code, K, B)
    peaks = measured_peaks()
    achieved = ab / (ms_step * 1e-3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (device AWGN, all-zero codeword)",
            "config": {"workload": "learned_qc_n7493", "frames_per_step": B, "iters": K, "params": list(beta.shape),
                       "ebn0_db": [1.5, 3.5], "step": "forward + BCE + adjoint + Adam", "phases": phases,
                       "l2": "flushed between timed steps (256 MB write)",
                       "value_meaning": "information bits of the frames trained per second"},
            "e2e": {"value": world * B * w.K / (e2e_ms / args.steps * 1e-3) / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": int(h_llr.numel() * 4), "d2h_bytes_per_step": 4},
            "gpu_launches": args.steps * (4 + 6 * K),  # forward 1 + 2K, loss 2, adjoint 4K, Adam 1
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                         "peak_source": peaks["source"] + " copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                         "algorithmic_bytes_per_launch": ab, "kernel": "training step (lf_*, bce, lb_*, adam)",
                         "kernel_ms": ms_step},
            "clocks": clocks}
    if not args.no_cpu_baseline:
        wl = I.make_workload("qc_n7493", n_frames=64, ebn0_db=2.5, zero_codeword=True)
        line["cpu_baseline"] = cpu_oracle_learned_sample(wl, K, float(os.environ.get("BENCH_CPU_BUDGET_S", "12")))
    print(json.dumps(line), flush=True)
    return 0


COMPARE_FORMS = ("ss_1bit", "ss_fixed", "two_scan", "two_scan_1bit")


def time_decode(ldpc, code, params, llr, F, flush, stream, dev, steps: int, warmup: int):
    """Mean device ms of ldpc_decode_batch over `steps` decodes after `warmup`,
    L2 flushed before each (outside the events)."""
    import torch
    ws_bytes = ldpc.ldpc_workspace_size(code.handle, params, F)
    N8 = (code.n_vars + 7) // 8
    bits = torch.empty((F, N8), dtype=torch.uint8, device=dev)
    iters = torch.empty(F, dtype=torch.int32, device=dev)
    ok = torch.empty(F, dtype=torch.uint8, device=dev)
    ws = torch.empty(max(ws_bytes, 1) + 256, dtype=torch.uint8, device=dev)
    ws_ptr = (ws.data_ptr() + 255) & ~255

    class _WS:
        def data_ptr(self):
            return ws_ptr

    def one():
        ldpc.ldpc_decode_batch(code.handle, params, llr, F, bits, iters, ok, None, _WS() if ws_bytes else None,
                               ws_bytes, stream)

    evs = []
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            one()
        for s in range(steps):
            flush.fill_(s & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            one()
            b.record(stream)
            evs.append((a, b))
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in evs])), bits, iters, ok


def compare_forms(ldpc, code, w, llr, F, main_form, flush, stream, dev, main_ms):
    """The other forms on the same frames and iterations: per-edge single scan,
    two-scan with per-edge messages, two-scan with the Section V state."""
    peaks = measured_peaks()
    out = {}
    K, iters_cap = w.K, w.params["max_iter"]
    for form in COMPARE_FORMS:
        if form == main_form:
            ms = main_ms
            chosen = ldpc.ldpc_kernel_choice(code.handle, ldpc.make_params(form=form, **w.params), F)
        else:
            params = ldpc.make_params(form=form, **w.params)
            try:
                chosen = ldpc.ldpc_kernel_choice(code.handle, params, F)
            except ldpc.LdpcError as e:
                out[form] = {"unavailable": str(e)}
                continue
            ms, _, it, _ = time_decode(ldpc, code, params, llr, F, flush, stream, dev, steps=5, warmup=2)
            assert int(it.min()) == iters_cap and int(it.max()) == iters_cap
        ab = algorithmic_bytes(w.code, form, iters_cap, F)
        out[form] = {"ms": ms, "value": F * K / (ms * 1e-3) / 1e9, "unit": UNIT, "kernel": chosen,
                     "hbm_frac": ab["per_launch"] / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                     "bytes_per_frame_iter": ab["per_frame_iter"]}
    ss = out.get("ss_1bit", {}).get("ms")
    if ss:
        out["two_scan_over_single_scan_time"] = {f: out[f]["ms"] / ss for f in ("two_scan", "two_scan_1bit")
                                                 if "ms" in out.get(f, {})}
    out["note"] = ("same frames, same fixed iteration count, early stop off, L2 flushed before each decode; "
                   "hbm_frac = the form's streaming-model bytes over its time and the copy bandwidth")
    return out


# Eb/N0 points (dB) of the FER curve the line carries, per workload: the
# workload's own channel point first, then the code's waterfall region.
FER_POINTS = {"irr_n64800": [1.0, 1.5, 2.0, 2.5, 3.0], "qc_n7493": [2.5, 2.75, 3.0],
              "reg36_n1008": [2.0, 2.5, 3.0]}


def fer_point(ldpc, code, w, llr, F, form, stream, dev, min_errors=100, max_frames=1 << 15):
    """Frame error rates of the benchmarked decoder (early stop on) at the
    stated Eb/N0 points: random codewords of the code (a pool from its encoder),
    BPSK over AWGN generated on the device, the int8 channel quantization of the
    workload; each point runs until min_errors frame errors or max_frames
    frames, with a Wilson 95 % interval."""
    import torch
    from paper_cs_0609090_gb300 import fer
    params = ldpc.make_params(form=form, **dict(w.params, early_stop=1))
    pool = fer.CodewordPool(w.code, 256, seed=12345, device=dev)
    run = fer.int8_decoder(code, params, w.delta, w.qc, F, dev)
    rate = (w.code.n_vars - w.code.n_checks) / w.code.n_vars
    pts = []
    for eb in FER_POINTS.get(w.name, [w.ebn0_db]):
        r = fer.run_point(run, w.code.n_vars, rate, eb, pool, min_errors=min_errors, max_frames=max_frames,
                          batch=F, seed=99)
        pts.append({k: r[k] for k in ("ebn0_db", "frames", "errors", "fer", "wilson95", "mean_iters")})
    torch.cuda.synchronize()
    return {"points": pts, "max_iter": w.params["max_iter"], "early_stop": 1, "form": form,
            "codewords": "random, pool of 256 from the code's encoder (seed 12345); device AWGN, seed 99",
            "stop": f">= {min_errors} frame errors or {max_frames} frames per point"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="irr_n64800")
    ap.add_argument("--form", default="ss_1bit", choices=["ss_1bit", "ss_fixed", "two_scan", "two_scan_1bit"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel", default="auto",
                    choices=["auto", "onchip_int", "onchip_half", "stream", "cluster", "persistent", "pingpong"])
    ap.add_argument("--dtype", default="int8", choices=["int8", "f32"])
    ap.add_argument("--schedule", default="flooding", choices=["flooding", "layered"],
                    help="layered: the single scan with column-disjoint layers updating in place")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the comparison forms and the FER measurement (profiling runs)")
    ap.add_argument("--frames", type=int, default=None,
                    help="decode this many frames of the workload instead of its batch (profiling runs)")
    ap.add_argument("--iters", type=int, default=None,
                    help="run this many iterations instead of the workload's (profiling runs)")
    ap.add_argument("--ebn0", type=float, default=None,
                    help="channel Eb/N0 in dB instead of the workload's (analysis runs)")
    ap.add_argument("--early-stop", action="store_true",
                    help="stop each frame at a codeword (analysis runs; the metric is quoted at fixed "
                         "iterations, so the line then reports the mean iterations too)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)

    if args.workload == "multi8":
        return run_multi(args, world, rank, local)
    if args.workload == "learned_qc_n7493":
        return run_learned(args, world, rank, local)

    import torch
    from paper_cs_0609090_gb300 import ldpc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = I.make_workload(args.workload, frame_seed=1 + rank, n_frames=args.frames, ebn0_db=args.ebn0)
    w.params["early_stop"] = 1 if args.early_stop else 0
    if args.iters is not None:
        w.params["max_iter"] = args.iters
    F, N, K = w.n_frames, w.code.n_vars, w.K
    code = ldpc.Code.from_inputs(w.code, device=local)
    wp = dict(w.params)
    if args.dtype == "f32":
        wp["dtype"] = "f32"
    params = ldpc.make_params(form=args.form, kernel=args.kernel, schedule=args.schedule, **wp)
    ws_bytes = ldpc.ldpc_workspace_size(code.handle, params, F)
    chosen = ldpc.ldpc_kernel_choice(code.handle, params, F)
    kname = kernel_name(args.form, args.dtype, args.schedule, chosen, ws_bytes, code)
    host_llr = w.q0 if args.dtype == "int8" else w.llr.astype(np.float32)
    llr = torch.from_numpy(host_llr).to(dev)
    bits = torch.empty((F, (N + 7) // 8), dtype=torch.uint8, device=dev)
    iters = torch.empty(F, dtype=torch.int32, device=dev)
    ok = torch.empty(F, dtype=torch.uint8, device=dev)
    ws = torch.empty(max(ws_bytes, 1) + 256, dtype=torch.uint8, device=dev)
    ws_ptr = (ws.data_ptr() + 255) & ~255
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # 256 MB > 129 MB L2

    class _WS:  # aligned workspace pointer for the binding
        def data_ptr(self):
            return ws_ptr

    def step():
        ldpc.ldpc_decode_batch(code.handle, params, llr, F, bits, iters, ok, None,
                               _WS() if ws_bytes else None, ws_bytes, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    # all frames ran the fixed iteration count
    if not args.early_stop:
        assert int(iters.min()) == w.params["max_iter"] and int(iters.max()) == w.params["max_iter"]
    mean_iters = float(iters.double().mean().item())

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.fill_(s & 0xff)  # evict L2 between timed steps (outside the event pair)
            evs[s][0].record(stream)
            step()
            evs[s][1].record(stream)
    torch.cuda.synchronize()
    dev_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = float(np.sum(dev_ms))

    # end to end through the C ABI: pinned host LLRs in, decisions/iters/flags out
    h_llr = torch.from_numpy(host_llr).pin_memory()
    h_bits = torch.empty_like(bits, device="cpu").pin_memory()
    h_iters = torch.empty_like(iters, device="cpu").pin_memory()
    h_ok = torch.empty_like(ok, device="cpu").pin_memory()
    e2e_evs = []
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.fill_(s & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            llr.copy_(h_llr, non_blocking=True)
            step()
            h_bits.copy_(bits, non_blocking=True)
            h_iters.copy_(iters, non_blocking=True)
            h_ok.copy_(ok, non_blocking=True)
            b.record(stream)
            e2e_evs.append((a, b))
    torch.cuda.synchronize()
    e2e_serial_ms = float(np.sum([a.elapsed_time(b) for a, b in e2e_evs]))

    # the same, pipelined as a server runs it: two input buffers and two output
    # sets; uploads on one stream and read-backs on another, so that step s+1's
    # host->device copy runs while step s decodes and step s-1's results come
    # back (a single copy stream would queue the upload behind the read-back,
    # which waits for the decode).  The L2 flush stays before every decode,
    # inside the timed region, timed from the first upload to the last
    # read-back.
    up, down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    llr_b = [llr, torch.empty_like(llr)]
    out_b = [(bits, iters, ok), (torch.empty_like(bits), torch.empty_like(iters), torch.empty_like(ok))]
    copied = [torch.cuda.Event() for _ in range(args.steps)]
    decoded = [torch.cuda.Event() for _ in range(args.steps)]
    read = [torch.cuda.Event() for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    up.wait_event(t0)
    for s in range(args.steps):
        b = s & 1
        with torch.cuda.stream(up):
            if s >= 2:
                up.wait_event(decoded[s - 2])  # buffer b's last reader
            llr_b[b].copy_(h_llr, non_blocking=True)
            copied[s].record(up)
        with torch.cuda.stream(stream):
            if s >= 2:
                stream.wait_event(read[s - 2])  # output set b read back
            flush.fill_(s & 0xff)
            stream.wait_event(copied[s])
            ob = out_b[b]
            ldpc.ldpc_decode_batch(code.handle, params, llr_b[b], F, ob[0], ob[1], ob[2], None,
                                   _WS() if ws_bytes else None, ws_bytes, stream)
            decoded[s].record(stream)
        with torch.cuda.stream(down):
            down.wait_event(decoded[s])
            h_bits.copy_(out_b[b][0], non_blocking=True)
            h_iters.copy_(out_b[b][1], non_blocking=True)
            h_ok.copy_(out_b[b][2], non_blocking=True)
            read[s].record(down)
    t1.record(down)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    e2e_ms = t0.elapsed_time(t1)
    if not args.early_stop:
        assert int(h_iters.min()) == w.params["max_iter"] and int(h_iters.max()) == w.params["max_iter"]

    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms, e2e_ms, e2e_serial_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms, e2e_ms, e2e_serial_ms = float(t[0]), float(t[1]), float(t[2])
        dist.barrier()
    if rank != 0:
        return 0

    ms_step = total_ms / args.steps
    value = world * F * K / (ms_step * 1e-3) / 1e9
    e2e_pipe = world * F * K / (e2e_ms / args.steps * 1e-3) / 1e9
    e2e_serial = world * F * K / (e2e_serial_ms / args.steps * 1e-3) / 1e9
    # both loops go through the C ABI with every copy inside the timed region;
    # the pipelined one wins once a step outlasts its extra stream and event
    # calls (about 0.5 ms), the serial one on shorter steps
    e2e_mode = "pipelined" if e2e_pipe >= e2e_serial else "serial"
    e2e_val = max(e2e_pipe, e2e_serial)
    roofline = roofline_line(kname, w, args.form, args.dtype, F, ms_step, clocks,
                             torch.cuda.get_device_properties(dev).multi_processor_count)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": w.name, "form": args.form, "n_frames": F, "iters": w.params["max_iter"],
                       "N": N, "M": w.code.n_checks, "E": w.code.n_edges, "K": K,
                       "ebn0_db": w.ebn0_db, "rule": w.params["rule"], "early_stop": w.params["early_stop"],
                       "mean_iters": mean_iters,
                       "l2": "flushed between timed steps (256 MB write)", "frames_per_rank": F,
                       "kernel": args.kernel, "kernel_chosen": chosen, "schedule": args.schedule},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(host_llr.nbytes),
                    "d2h_bytes_per_step": int(bits.numel() + iters.numel() * 4 + ok.numel()),
                    "mode": e2e_mode, "pipelined_value": e2e_pipe, "serial_value": e2e_serial,
                    "pipeline": "upload and read-back streams: step s+1's input copy overlaps step s's decode"},
            "gpu_launches": args.steps * (1 if (ws_bytes == 0 or args.schedule == "layered")
                                          else 2 if kname == "pp_kernel"
                                          else 3 + w.params["max_iter"] if kname == "pp2_rows"
                                          else 3 + 2 * w.params["max_iter"]),
            "roofline": roofline, "clocks": clocks}
    if not args.no_compare and args.dtype == "int8" and args.schedule == "flooding" and world == 1:
        line["comparisons"] = compare_forms(ldpc, code, w, llr, F, args.form, flush, stream, dev, ms_step)
        line["fer"] = fer_point(ldpc, code, w, llr, F, args.form, stream, dev)
    if not args.no_cpu_baseline and args.dtype == "int8":
        lay = ldpc.ldpc_code_layers(code.handle, w.code.n_checks)[1] if args.schedule == "layered" else None
        info, _ = cpu_oracle_sample(w, args.form, budget_s=float(os.environ.get("BENCH_CPU_BUDGET_S", "12")),
                                    max_frames=F, layers=lay)
        line["cpu_baseline"] = info
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
