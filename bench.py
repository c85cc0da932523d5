#!/usr/bin/env python
"""Throughput of the exactly K-sparse sFFT-DT hot path on GB300.

Workload (one "step"): one batch of B independent seeded synthetic signals,
N = 2^22 complex64, K = 4096 non-zero frequencies at uniform positions with
|X| ~ U[1, 10] and uniform phase, transformed by iterative sFFT-DT
(Algorithm 1) with d = 512 (M = 2^13 bins), a_m = 4 levels, FP32
(compensated) FFTs and FP64 solves -- through the C ABI (sft_exact).

Printed: one JSON line (rank 0) with signals/s, the end-to-end rate through
the host entry point (sft_exact_host, pinned buffers, copies timed), the
roofline of the dominant kernel, sampled SM clocks, recovered fraction and
the error against the FP64 oracle on a sample, and the oracle's own rate on
the host cores as a CPU baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B]
  python bench.py --impl reference ...   # the FP64 CPU oracle as reference arm
Multi-GPU (torchrun, one process per GPU): every rank transforms its own
batch (replicas, no data-path collective); value = all signals / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import siggen  # noqa: E402

N, K, M = 1 << 22, 4096, 1 << 13
D = N // M
METRIC = "SFT signals/sec at N=2^22,K=4096; recovered fraction; max err vs FP64 oracle"
WORKLOAD = "exact-iter N=2^22 K=4096 d=512 (M=2^13) a_m=4 c64 |X|~U[1,10]"
THROTTLE = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=152)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    return ap.parse_args()


# ------------------------------------------------------------------ utilities
def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def gen_batch(B, seed0, threads):
    out = np.empty((B, N), np.complex64)
    supps = [None] * B

    def one(i):
        x, s, _ = siggen.exact_signal(N, K, seed0 + i, mag=(1, 10), dtype=np.complex64)
        out[i] = x
        supps[i] = s

    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, range(B)))
    return out, supps


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons, sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [t.strip() for t in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1407_8315_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """dram bytes per launch of `kernel` from the committed ncu summary, or
    None if the summary is missing or was taken on other kernel sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    ent = t.get(kernel)
    if not ent or ent.get("source_sha") != source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


# Algorithmic work per launch of each stage, per signal.  The gather/FFT
# stages must read 2 shifts x M_l samples of 8 B (complex64) and produce
# 2 x M_l syndromes; bytes below count the samples (the input the method has
# to touch).  FP32 work of the compensated FFT: 5 M log2 M flop per shift
# counted as real flops of a radix-2 FFT.
def stage_model(name):
    if name.startswith("gather_fft_l"):
        l = int(name[-1])
        Ml = M >> l
        return {"bytes": 2 * Ml * 8, "flops": 2 * 5 * Ml * int(np.log2(Ml))}
    return None


def kernel_of(stage: str) -> str:
    """The __global__ function (template instance) that runs a stage: one
    gather/FFT kernel serves every level, the fold and decode kernels are
    instantiated per level (a = l + 1)."""
    if stage.startswith("gather_fft"):
        return "k_gather_fft"
    if stage.startswith("fold_l"):
        return f"k_iter_fold<a={int(stage[-1]) + 1}>"
    if stage.startswith("decode_l"):
        return f"k_iter_decode<a={int(stage[-1]) + 1}>"
    return "k_" + stage


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1407_8315_gb300 import Plan, build

    ws, rank, local = dist_setup(args)
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build()
    B = args.batch
    threads = max(1, min(16, os.cpu_count() or 1))
    x_host_np, supps = gen_batch(B, 1_000_000 * (rank + 1), threads)
    # pinned host copy for the end-to-end leg
    pinned = torch.empty((B, N), dtype=torch.complex64, pin_memory=True)
    pinned.numpy()[:] = x_host_np
    x_dev = pinned.to("cuda", non_blocking=False)
    plan = Plan(N, K, D, "iter", "mixed", max_signals=B)
    cap = 2 * K
    out = plan.exact(x_dev, cap)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.exact(x_dev, cap, out)
    torch.cuda.synchronize()

    # ---- timed region: K steps, device time by CUDA events, stage events live
    plan.set_profiling(True)
    _ = plan.stage_times()  # reset
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.exact(x_dev, cap, out)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    stages = plan.stage_times()
    plan.set_profiling(False)
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / args.steps
    value = ws * B * args.steps / (ms / 1e3)
    launches = plan.launches_per_call * args.steps

    # ---- quality on this rank's batch: recovered fraction vs planted support
    cnt = out.count.cpu().numpy()
    idx = out.idx.cpu().numpy()
    found = sum(int(np.isin(idx[b, :cnt[b]], supps[b]).sum()) for b in range(B))
    false_pos = sum(int(cnt[b]) for b in range(B)) - found
    recovered = found / (B * K)

    # ---- end to end through the host entry point.  Two page-locked copies
    # of the batch alternate so that no line of one step's input can still
    # sit in L2 at the next step; the kernels read the samples in place over
    # NVLink-C2C and write the results into page-locked host arrays.
    import paper_1407_8315_gb300.sft as S
    pinned2 = torch.empty((B, N), dtype=torch.complex64, pin_memory=True)
    pinned2.numpy()[:] = x_host_np
    srcs = [pinned.numpy(), pinned2.numpy()]
    h_out = S.Result(torch.empty((B, cap), dtype=torch.int64, pin_memory=True).numpy(),
                     torch.empty((B, cap), dtype=torch.complex128, pin_memory=True).numpy(),
                     torch.empty(B, dtype=torch.int64, pin_memory=True).numpy(),
                     torch.empty(B, dtype=torch.int32, pin_memory=True).numpy(),
                     torch.empty(B, dtype=torch.int32, pin_memory=True).numpy())
    for i in range(3):
        plan.exact_host(srcs[i & 1], cap, h_out)  # warm
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(args.e2e_steps):
        plan.exact_host(srcs[i & 1], cap, h_out)
    e2e_s = time.perf_counter() - t0
    if ws > 1:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    # bytes crossing the host link per step: the samples of the shifts the
    # transform reads (2 shifts x M_l samples of 8 B at each level) in, the
    # recovered entries and per-signal counters out
    levels = 4
    h2d = int(B * sum(2 * (M >> l) * 8 for l in range(levels)))
    d2h = int(int(h_out.count.sum()) * 24 + B * 16)
    e2e = {"value": ws * B * args.e2e_steps / e2e_s, "unit": "signals/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "path": "sft_exact_host, page-locked host input read in place (zero-copy gather "
                   "over NVLink-C2C), results written in place; two alternating input copies"}

    if ws > 1:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (live stage events).  Stages are
    # grouped by the kernel that runs them (k_gather_fft serves every level);
    # the dominant kernel is the one with the largest share of step time.
    peaks, peak_src = measured_peaks()
    groups = {}
    for name, (ms_tot, nl) in stages.items():
        kern = kernel_of(name)
        g = groups.setdefault(kern, {"ms": 0.0, "launches": 0, "bytes": 0, "stages": []})
        g["ms"] += ms_tot
        g["launches"] += nl
        g["stages"].append(name)
        model = stage_model(name)
        if model is not None:
            g["bytes"] += model["bytes"] * B * nl
    dom_name = max(groups, key=lambda k: groups[k]["ms"])
    dom = groups[dom_name]
    step_ms = sum(g["ms"] for g in groups.values())
    if dom["bytes"]:
        ach = dom["bytes"] / (dom["ms"] / 1e3) / 1e9
        roof = {"kernel": dom_name, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "peak_source": peak_src,
                "traffic": ncu_traffic(dom_name), "share": dom["ms"] / step_ms,
                "ms_per_launch": dom["ms"] / dom["launches"]}
    else:
        roof = {"kernel": dom_name, "bound": "alu", "achieved": None, "peak": None,
                "unit": None, "frac": None, "peak_source": peak_src, "traffic": None,
                "share": dom["ms"] / step_ms, "ms_per_launch": dom["ms"] / dom["launches"]}
    stage_ms = {k: round(v[0] / v[1], 5) for k, v in stages.items()}

    # ---- CPU baseline and error vs the FP64 oracle on a sample
    cpu = None
    err = {"max_rel_err": None, "support_mismatch_signals": None, "sample_signals": 0}
    if not args.no_cpu:
        cpu, err = cpu_baseline(x_host_np, idx, out.val.cpu().numpy(), cnt, plan, args.cpu_seconds)

    line = {
        "metric": METRIC, "value": value, "unit": "signals/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "ff32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch_per_gpu": B, "mode": "iter",
                   "precision": "mixed (compensated-FP32 FFT, FP64 solves)",
                   "parallelism": f"replicas x{ws}",
                   "l2": f"inputs larger than L2 ({B} x 32 MiB per GPU), no flush"},
        "recovered_fraction": recovered, "false_positives": false_pos,
        "vs_oracle": err,
        "e2e": e2e, "gpu_launches": launches, "stage_ms_per_launch": stage_ms,
        "roofline": roof, "clocks": clk, "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def cpu_baseline(xs, idx, val, cnt, plan, seconds):
    """Time the FP64 oracle (as it stands) on the host cores over signals of
    the benchmark batch, and compare its output with the GPU's."""
    import oracle
    oracle.build()
    p = plan.params
    tol = dict(zero_tol=p.zero_tol, root_tol=p.root_tol, res_tol=p.res_tol)
    cores = os.cpu_count() or 1
    B = xs.shape[0]

    def one(b):
        return b, oracle.exact(xs[b], M, 4, oracle.ITER, max_iters=4, cap=2 * K, **tol)

    results = {}
    done = 0
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        while True:
            for b, r in ex.map(one, range(B)):
                results[b] = r
                done += 1
            if time.perf_counter() - t0 >= seconds or done >= 8 * B:
                break
    el = time.perf_counter() - t0
    worst, mism = 0.0, 0
    for b, (oi, ov, ou) in results.items():
        gi, gv = idx[b, :cnt[b]], val[b, :cnt[b]]
        o = np.argsort(gi, kind="stable")
        gi, gv = gi[o], gv[o]
        if not np.array_equal(gi, oi):
            mism += 1
            continue
        if len(oi):
            worst = max(worst, float((np.abs(gv - ov) / np.abs(ov)).max()))
    cpu = {"value": done / el, "unit": "signals/s", "cores": cores, "kind": "oracle",
           "sample": f"{done} transforms of the {B} benchmark signals ({len(results)} distinct), "
                     f"one per thread, {cores} threads, {el:.1f} s"}
    err = {"max_rel_err": worst, "support_mismatch_signals": mism, "sample_signals": len(results)}
    return cpu, err


# ------------------------------------------------------------ reference arm
def run_reference(args):
    """The FP64 CPU oracle on the host cores: each step transforms one signal
    per core (a bounded sample of the same workload)."""
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    xs, _ = gen_batch(cores, 7_000_000, max(1, min(16, cores)))
    tol = oracle.TOL_MIXED

    def one(b):
        return oracle.exact(xs[b], M, 4, oracle.ITER, max_iters=4, cap=2 * K, **tol)

    with ThreadPoolExecutor(max_workers=cores) as ex:
        for _ in range(args.warmup):
            list(ex.map(one, range(cores)))
        t0 = time.perf_counter()
        for _ in range(args.steps):
            list(ex.map(one, range(cores)))
        el = time.perf_counter() - t0
    value = cores * args.steps / el
    line = {
        "metric": METRIC, "value": value, "unit": "signals/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "batch_per_step": cores, "mode": "iter",
                   "precision": "FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": "signals/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} signals per step, one per thread"},
        "e2e": {"value": value, "unit": "signals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
