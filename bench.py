#!/usr/bin/env python
"""Benchmark of the EnSF analysis step on GB300.

One "step" is one full analysis (Sec. III-A.2): row norms and splits of the
forecast ensemble, the initial Gaussian particles, then K Euler-Maruyama steps
of Gram + softmax + weighted sum + score + update.  Metric: member-steps/s =
N * K / (wall time of one analysis).  With several GPUs (torchrun) one filter
is split along the state dimension over the GPUs (strong scaling); with
--replicas every GPU runs its own filter and the ranks' member-steps add up
(weak scaling).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--path split-bf16|split|fp32] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (rows are independent, so a few particle rows
through a few Euler-Maruyama steps is an exact sample of the work).
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

from paper_2407_12168_gb300 import inputs  # noqa: E402

PATHS = {
    # name: (gram precision, W X precision)
    "split-bf16": ("split", "bf16"),
    "split": ("split", "split"),
    "fp32": ("fp32", "fp32"),
    "tf32-bf16": ("tf32", "bf16"),   # precision study: TF32 Gram
    "tf32": ("tf32", "split"),       # precision study: TF32 Gram, split W X (isolates the Gram's error)
    "bf16": ("bf16", "bf16"),        # precision study: one BF16 product in both contractions
}
METRIC = "EnSF member-steps/s (analysis step, K Euler-Maruyama steps per member)"
UNIT = "member-steps/s"
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max clock


def _dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), \
        int(os.environ.get("WORLD_SIZE", "1"))


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of per-rank timings (every rank gets the result);
    with no process group the values come back unchanged."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def _traffic_record(kernel: str, workload: str, path: str, splits: int = 0, n: int = 0):
    """DRAM traffic per launch from a committed ncu summary, valid only while
    the kernel source is unchanged (sha256 of the kernel file and its PTX
    wrappers, recorded beside the number)."""
    fn = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(fn):
        return None
    csrc = os.path.join(ROOT, "paper_2407_12168_gb300", "csrc")
    srcs = ["ensf_simt.cu"] if path == "fp32" else ["ensf_tc.cu", "ensf_ptx.cuh"]
    h = hashlib.sha256()
    for f in srcs:
        h.update(open(os.path.join(csrc, f), "rb").read())
    sha = h.hexdigest()[:16]
    for line in open(fn):
        m = re.match(r"^traffic\s+(\S+)\s+(\S+)\s+(\S+)\s+(\S+)\s+bytes_per_launch=(\d+)(?:\s+splits=(\d+))?",
                     line)
        if m and m.group(1) == kernel and m.group(2) == workload and m.group(3) == path and m.group(4) == sha:
            traffic = int(m.group(5))
            if m.group(6) and splits and n:
                # the Gram's FP32 partials: S x N^2 x 4 B, written once per launch
                traffic += (int(splits) - int(m.group(6))) * n * n * 4
            return traffic
    return None


def _traffic_for(kernel: str, p, args):
    """The recorded traffic, when this run launched the kernel in the shape it
    was captured in: the CTA-pair Gram on BF16 planes (with or without the
    next step's noise written by its spare warps), W X in tiles of 256
    particles (reading the noise slice, or with the TMA-staged epilogue
    that draws the noise itself)."""
    t = args.tuning or {}
    inline = bool(t.get("noise_inline") == 1 or args.inline_noise)
    if kernel == "gram":
        if t.get("gram_cta_pair") != 1 or t.get("gram_fp32_particles") or t.get("gram_fused_softmax") or \
                t.get("noise_inline") == 2:
            return None
        tag = "gram_pair" if inline else "gram_pair_noise"
    elif kernel == "wx_em":
        if t.get("wx_tile_n") != 256 or t.get("noise_inline") == 2:
            return None
        tag = "wx_em_staged" if inline else "wx_em_slice"
    else:
        return None
    return _traffic_record(tag, p.name, args.path, t.get("gram_splits") or 0, p.n)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_problem(workload: str, rank: int):
    if workload == "batched-uneven":  # the reference arm samples the first filter of the batch
        return inputs.batched_uneven(seed=3 + 1000 * rank)[0]
    fn = inputs.WORKLOADS[workload]
    # every rank runs an independent filter (another seed: another truth, prior, noise)
    return fn(seed={"plain-64": 1, "sparse-arctan-128": 2, "large-512": 4, "medium-192": 5}[workload] + 1000 * rank)


def cpu_baseline(p, budget_s: float = 15.0, J: int = 0):
    """The FP64 oracle as it stands on the host cores, on a bounded sample of
    the workload: `rows` particle rows through the first `k_stop` of the K
    Euler-Maruyama steps (rows are independent, every step costs the same).
    With J, the oracle's mini-batch form over an identity permutation (the
    cost of a step does not depend on which members the window holds)."""
    from oracle import oracle as o
    mb = dict(perm=np.arange(p.n), J=J) if J else {}
    t0 = time.perf_counter()
    o.analysis(p.prior, p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed, rows=[0], k_stop=1, **mb)
    per = max(time.perf_counter() - t0, 1e-4)
    k_stop = int(max(1, min(p.K, budget_s / per)))
    rows = int(max(1, min(p.n, budget_s / (per * k_stop))))
    t0 = time.perf_counter()
    out = o.analysis(p.prior, p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed,
                     rows=list(range(rows)), k_stop=k_stop, **mb)
    dt = time.perf_counter() - t0
    rec = {"value": rows * k_stop / dt, "unit": UNIT, "cores": o.num_threads(), "kind": "oracle",
           "sample": f"{rows} particle row(s) x {k_stop} of {p.K} Euler-Maruyama steps of {p.name} "
                     f"(N={p.n}, d={p.d}{f', J={J}' if J else ''}), {dt:.1f} s"}
    # when the sample is the whole analysis, its ensemble is the FP64 answer
    return rec, (out if rows == p.n and k_stop == p.K else None)


def run_reference(args):
    rank, _, world = _dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as o
    p = make_problem(args.workload, 0)
    t0 = time.perf_counter()
    o.analysis(p.prior, p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed, rows=[0], k_stop=1)
    per = max(time.perf_counter() - t0, 1e-4)
    k_stop = int(max(1, min(p.K, args.ref_step_s / per)))
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o.analysis(p.prior, p.y, p.mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed, rows=[it % p.n],
                   k_stop=k_stop)
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = float(np.sum(times))
    value = args.steps * k_stop / tot
    sample = f"1 particle row x {k_stop} of {p.K} Euler-Maruyama steps of {p.name} (N={p.n}, d={p.d}) per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(p, "oracle-fp64", world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": o.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _config(p, path, world):
    return {"workload": p.name, "N": p.n, "d": p.d, "K": p.K, "eps": p.eps, "sigma_obs": p.sigma_obs,
            "obs": ("arctan" if p.obs_op == 1 else "identity") + ("" if p.mask is None else
                                                                  f", {int(p.mask.sum())} of {p.d} points"),
            "path": path, "noise": "Philox4x32-10 in-kernel",
            "l2": "inputs larger than L2" if p.n * p.d * 4 > 256 << 20 else "L2 flushed between steps",
            "parallelism": f"{world} independent filter(s), one per GPU"}


def _roofline(kernel, rec, p, gram, wx, args, peaks):
    """Roofline entry of one kernel kind from its event-timed launches.

    gram (Z X^T, 2 N^2 d FLOP algorithmic per launch; split-BF16x3 executes
    three BF16 products) is a dense contraction: tensor (or FP32 ALU) bound.
    wx_em (W X + score + Euler-Maruyama) moves per launch 8 N d bytes of
    particle state (read + write), 4 N d of noise when it reads a
    pre-generated slice (none when it draws the noise itself), 2 N d of X^T
    (BF16), and 4 N d of BF16 Z planes when the Gram runs on tensor cores: at
    N = 1024 its 2 N^2 d FLOP sit below the BF16 ridge, so it is HBM bound."""
    launches, timed, tot_ms = rec
    avg_ms = tot_ms / timed
    n, d = p.n, p.d
    nx = args.minibatch or n          # members in the prior-score sum of one step
    prec = gram if kernel == "gram" else wx
    flops = 2.0 * n * nx * d
    if kernel == "wx_em" and prec != "fp32":
        # the noise slice is read only when the draws were made before W X;
        # drawn in its epilogue they cost instructions, not bytes
        t = args.tuning or {}
        slice_read = not (t.get("noise_inline") == 1 or args.inline_noise)
        nbytes = ((8 + (4 if slice_read else 0) + (4 if gram != "fp32" else 0)) * n * d
                  + 2 * (2 if prec == "split" else 1) * nx * d + 5 * d)
        peak = float(peaks["hbm_gbs"]) if peaks else 6800.0
        achieved = nbytes / (avg_ms / 1e3) / 1e9
        return {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": _traffic_for(kernel, p, args),
                "peak_source": "measured HBM copy (MEASURED_PEAKS.json)" if peaks else "fallback",
                "algorithmic_bytes_per_launch": nbytes, "avg_launch_ms": avg_ms,
                "tflops": flops / (avg_ms / 1e3) / 1e12}
    if kernel == "softmax_rows":
        # split-K partials read (FP32), weights written (BF16 planes or FP32), FP64 norms read
        splits = (args.tuning or {}).get("gram_splits") or 1
        w_bytes = 4 if wx == "fp32" else (4 if wx == "split" else 2)
        nbytes = (4 * splits + w_bytes) * n * nx + 8 * nx
        peak = float(peaks["hbm_gbs"]) if peaks else 6800.0
        achieved = nbytes / (avg_ms / 1e3) / 1e9
        return {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": "measured HBM copy (MEASURED_PEAKS.json)" if peaks else "fallback",
                "algorithmic_bytes_per_launch": nbytes, "avg_launch_ms": avg_ms,
                "note": "latency bound at this size (partials mostly L2-resident)"}
    if kernel not in ("gram", "wx_em"):
        return {"kernel": kernel, "bound": None, "avg_launch_ms": avg_ms}
    split_factor = {"split": 3.0, "bf16": 1.0, "fp32": 1.0, "tf32": 1.0}[prec]
    executed = flops * split_factor
    if prec == "fp32":
        bound, peak, src = "alu", FP32_SIMT_PEAK_TFLOPS, "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"
    else:
        bound = "tensor"
        if peaks:
            peak, src = float(peaks["bf16_tflops_sustained"]), "measured bf16 sustained (MEASURED_PEAKS.json)"
        else:
            peak, src = 1700.0, "fallback bf16 sustained"
        if prec == "tf32":  # TF32 dense is half the BF16 rate (1.1 of 2.25 PFLOP/s nominal)
            peak, src = peak * 1.1 / 2.25, src + " x 1.1/2.25 (nominal TF32/BF16 ratio)"
    achieved = flops / (avg_ms / 1e3) / 1e12
    return {"kernel": kernel, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": _traffic_for(kernel, p, args), "peak_source": src,
            "algorithmic_flops_per_launch": flops, "avg_launch_ms": avg_ms,
            "executed_flops_per_launch": executed, "executed_tflops": executed / (avg_ms / 1e3) / 1e12,
            "executed_frac": executed / (avg_ms / 1e3) / 1e12 / peak}


def _warm_host_copies(ensf, stream, ce_copies, sm_copies, rounds: int = 6):
    """Untimed rounds of the host<->device copies a timed region will make
    (dst.copy_(src) on the copy engines, ensf.copy_sm on the SMs), repeated
    until two consecutive rounds agree within 1.3x (the copies have settled);
    returns the rounds' times in ms."""
    import torch
    warm = []
    for _ in range(rounds):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for dst, src in ce_copies:
            dst.copy_(src, non_blocking=True)
        for dst, src in sm_copies:
            ensf.copy_sm(dst, src, 152)
        b.record(stream)
        torch.cuda.synchronize()
        warm.append(round(a.elapsed_time(b), 1))
        if len(warm) >= 2 and max(warm[-2:]) <= 1.3 * min(warm[-2:]):
            break
    return warm


def _cpu_nodes():
    """NUMA nodes whose CPUs this process may run on (from sysfs)."""
    import glob
    try:
        allowed = os.sched_getaffinity(0)
    except AttributeError:
        return None
    nodes = []
    for path in sorted(glob.glob("/sys/devices/system/node/node[0-9]*/cpulist")):
        cpus = set()
        for part in open(path).read().strip().split(","):
            if part:
                lo, _, hi = part.partition("-")
                cpus.update(range(int(lo), int(hi or lo) + 1))
        if cpus & allowed:
            nodes.append(int(path.split("/node")[-1].split("/")[0]))
    return nodes


def _host_buffers(ensf, p, small_pages=False, any_node=False):
    """Page-locked host copies of the inputs and a host buffer for the result
    (ensf_host_alloc: huge pages unless small_pages, on the device's nearest
    host NUMA node unless any_node), and a record of how much of them the
    kernel backs with huge pages and where their pages sit."""
    import torch
    huge, near = not small_pages, not any_node
    h_prior = ensf.host_empty(p.prior.shape, torch.float32, huge, near)
    h_prior.copy_(torch.from_numpy(p.prior))
    h_y = ensf.host_empty(p.y.shape, torch.float32, huge, near)
    h_y.copy_(torch.from_numpy(p.y))
    h_mask = None
    if p.mask is not None:
        h_mask = ensf.host_empty(p.mask.shape, torch.uint8, huge, near)
        h_mask.copy_(torch.from_numpy(p.mask))
    h_out = ensf.host_empty(p.prior.shape, torch.float32, huge, near)
    rec = {"alloc": "ensf_host_alloc" + ("" if huge else " (small pages)") + ("" if near else " (any node)")}
    try:
        rec["huge_page_fraction"] = {"prior": round(ensf.host_huge_fraction(h_prior), 3),
                                     "out": round(ensf.host_huge_fraction(h_out), 3)}
    except Exception as e:  # no smaps: the buffers are still page-locked
        rec["huge_page_fraction"] = str(e)
    (n_prior, dev_node), (n_out, _) = ensf.host_numa(h_prior), ensf.host_numa(h_out)
    rec["numa"] = {"prior": n_prior, "out": n_out, "device_nearest": dev_node, "process_cpus_on": _cpu_nodes()}
    return h_prior, h_y, h_mask, h_out, rec


def run_batched(args):
    """64 independent filters with uneven N and d (K = 50).  split paths: one
    batched launch per stage for all filters; fp32: one analysis call per
    filter (the plain one-launch-per-instance path)."""
    import torch
    rank, local_rank, world = _dist_env()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2407_12168_gb300 import ensf
    gram, wx = PATHS[args.path]
    probs = inputs.batched_uneven(seed=3 + 1000 * rank)
    K, eps = probs[0].K, probs[0].eps
    dev = torch.device("cuda", local_rank)
    filters = [dict(prior=torch.from_numpy(p.prior).to(dev), y=torch.from_numpy(p.y).to(dev),
                    mask=torch.from_numpy(p.mask).to(dev) if p.mask is not None else None,
                    sigma_obs=p.sigma_obs, obs_op=p.obs_op, seed=p.seed) for p in probs]
    outs = [torch.empty_like(f["prior"]) for f in filters]
    max_n, max_d = max(p.n for p in probs), max(p.d for p in probs)
    batch_tuning = None
    if gram == "fp32":
        handles = [ensf.Filter(p.n, p.d, gram="fp32", wx="fp32", graph=args.graph) for p in probs]

        def one(sd):
            for f, fl, o in zip(handles, filters, outs):
                f.analysis(fl["prior"], fl["y"], fl["mask"], fl["sigma_obs"], K, eps, fl["obs_op"],
                           seed=fl["seed"] + sd, out=o)
        prof_handles = handles
    else:
        h = ensf.Filter(max_n, max_d, gram=gram, wx=wx, graph=args.graph)
        # the k-range per batched Gram work item, timed on these filters
        batch_tuning = h.autotune_batched(filters, eps)

        def one(sd):
            h.analysis_batched([dict(fl, seed=fl["seed"] + sd) for fl in filters], K, eps, outs=outs)
        prof_handles = [h]
    stream = torch.cuda.current_stream()
    for w in range(args.warmup):
        one(w)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for s_ in range(args.steps):
            ev[s_][0].record(stream)
            one(100 + s_)
            ev[s_][1].record(stream)
        torch.cuda.synchronize()
    ms = float(sum(a.elapsed_time(b) for a, b in ev)) / args.steps
    for f in prof_handles:
        f.profile_enable(True)
    for s_ in range(args.steps):
        one(100 + s_)
    torch.cuda.synchronize()
    prof = {}
    for f in prof_handles:
        for k, v in f.profile_read().items():
            a = prof.get(k, (0, 0, 0.0))
            prof[k] = (a[0] + v[0], a[1] + v[1], a[2] + v[2])
        f.profile_enable(False)
    ms, = max_over_ranks([ms], dist, dev)
    if dist and rank != 0:
        dist.destroy_process_group()
        return 0
    member_steps = sum(p.n for p in probs) * K
    flops = sum(2.0 * p.n * p.n * p.d for p in probs)
    kern = {k: {"launches": v[0] // args.steps, "avg_ms": (v[2] / v[1]) if v[1] else None} for k, v in prof.items()}
    peaks = _peaks()
    # Gram time per Euler-Maruyama step (all filters): one batched launch, or one launch per filter
    gram_ms = prof["gram"][2] / (args.steps * K) if "gram" in prof and prof["gram"][1] else None
    roof = None
    if gram_ms:
        per_step_gram_ms = gram_ms
        peak = float(peaks["bf16_tflops_sustained"]) if peaks and gram != "fp32" else FP32_SIMT_PEAK_TFLOPS
        ach = flops / (per_step_gram_ms / 1e3) / 1e12
        roof = {"kernel": "gram", "bound": "tensor" if gram != "fp32" else "alu", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                "algorithmic_flops_per_step": flops, "gram_ms_per_step": per_step_gram_ms,
                "note": "latency-bound sizes: the Gram of all 64 filters per Euler-Maruyama step"}
    line = {"metric": METRIC, "value": world * member_steps / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"split-bf16": "bf16x3+bf16 (fp32 acc)", "split": "bf16x3 (fp32 acc)", "fp32": "f32"}[args.path],
            "data": "synthetic",
            "config": {"workload": "batched-uneven", "filters": len(probs), "K": K,
                       "N": sorted(set(p.n for p in probs)), "d": sorted(set(p.d for p in probs)),
                       "path": args.path + (" (one batched launch per stage)" if gram != "fp32"
                                            else " (one analysis call per filter)"),
                       "l2": "working set partly L2-resident (small filters)", "cuda_graph": args.graph,
                       "parallelism": f"{world} independent batch(es), one per GPU"},
            "roofline": roof, "kernels": kern, "gpu_launches": int(sum(v[0] for v in prof.values()) // args.steps),
            "clocks": clk.summary(), "tuning": batch_tuning}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def run_ours(args):
    import torch
    rank, local_rank, world = _dist_env()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2407_12168_gb300 import ensf

    gram, wx = PATHS[args.path]
    p = make_problem(args.workload, rank)
    dev = torch.device("cuda", local_rank)
    prior = torch.from_numpy(p.prior).to(dev)
    y = torch.from_numpy(p.y).to(dev)
    mask = torch.from_numpy(p.mask).to(dev) if p.mask is not None else None
    out = torch.empty_like(prior)
    f = ensf.Filter(p.n, p.d, gram=gram, wx=wx, graph=args.graph, inline_noise=args.inline_noise,
                    persistent=args.persistent)
    stream = torch.cuda.current_stream()
    tuning = None
    if args.set_tuning:
        # fixed launch shapes (no autotuner launches before the measured ones)
        tuning = dict(json.loads(args.set_tuning))
        f.set_tuning(p.n, p.d, **tuning)
    elif gram != "fp32" or wx != "fp32":
        tuning = f.autotune(prior, y, mask, p.sigma_obs, p.eps, p.obs_op, seed=p.seed, out=out)
    args.tuning = tuning
    small = p.n * p.d * 4 <= 256 << 20
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if small else None

    J = args.minibatch
    if J:
        if gram == "fp32":
            raise SystemExit("--minibatch needs a tensor-core path (split-bf16 or split)")
        # one seeded member permutation per analysis, drawn on the host and
        # made resident before any timed region
        perms = {}

        def perm_for(k_seed):
            if k_seed not in perms:
                g = np.random.default_rng([p.seed, 7, k_seed])
                perms[k_seed] = torch.from_numpy(g.permutation(p.n).astype(np.int32)).to(dev)
            return perms[k_seed]
        for k_seed in list(range(args.warmup)) + [100 + s_ for s_ in range(args.steps)] + \
                [200 + s_ for s_ in range(3)]:
            perm_for(k_seed)

    def analyse(pr, yy, mm, k_seed):
        if J:
            f.analysis_minibatch(pr, yy, mm, p.sigma_obs, p.K, p.eps, perm_for(k_seed), J, p.obs_op,
                                 seed=p.seed + k_seed, out=out)
        else:
            f.analysis(pr, yy, mm, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed + k_seed, out=out)

    def one(k_seed):
        analyse(prior, y, mask, k_seed)

    for w in range(args.warmup):
        one(w)
    torch.cuda.synchronize()

    # ---- end-to-end buffers: page-locked host copies of the inputs and the
    # result, backed by huge pages (ensf_host_alloc; buffers pinned page by
    # page copied 3-6x slower right after an analysis on a host that had been
    # busy) ----
    h_prior, h_y, h_mask, h_out, host_huge = _host_buffers(ensf, p, args.small_pages, args.any_node)
    d_prior, d_y = torch.empty_like(prior), torch.empty_like(y)
    d_mask = torch.empty_like(mask) if mask is not None else None
    # sequential end-to-end steps (copy in, analyse, copy out, the host takes
    # the result): the end-to-end figure of the mini-batch form, and for the
    # other forms one step that shows the raw copy times
    pipelined = not J
    e2e_steps = 1 if pipelined else max(1, min(args.steps, 3))
    ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    # the inner boundaries: inputs on the device, analysis done
    ei = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    # pipelined end-to-end steps (Filter.analyses_from_host): the copies of
    # analysis s +/- 1 overlap analysis s
    pipe_steps = max(3, min(args.steps, 8))
    h_out2 = ensf.host_empty(p.prior.shape, torch.float32, not args.small_pages) if pipelined else None
    copy_stream = torch.cuda.Stream() if pipelined else None
    # untimed passes first, as the device steps have their warm-up: the first
    # device writes into freshly pinned host pages cost a one-time mapping,
    # and after other processes on the host have freed much memory the first
    # gigabytes of host<->device copies run up to 80x slower (measured: a
    # 2 GiB copy-out took 927, 76, then 11 ms), recovering with the bytes
    # moved, not with time.  So the copies the timed region makes (copy
    # engines, and the SM copy of the first copy-in and last copy-out) are
    # repeated until two consecutive rounds agree within 1.3x (at most six
    # rounds); the rounds' times are reported.
    ce = [(d_prior, h_prior), (h_out, d_prior)] + ([(h_out2, d_prior)] if h_out2 is not None else [])
    warm = _warm_host_copies(ensf, stream, ce, [(h_out, out), (d_prior, h_prior)])

    def e2e_pipelined():
        jobs = [dict(prior=h_prior, y=h_y, mask=h_mask, out=(h_out, h_out2)[i % 2], seed=p.seed + 300 + i)
                for i in range(pipe_steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        evs = f.analyses_from_host(jobs, p.sigma_obs, p.K, p.eps, p.obs_op, stream=stream,
                                   copy_stream=copy_stream)
        t1.record(stream)
        return t0, t1, evs

    def e2e_step(s_):
        """One analysis through host buffers: host-to-device copies of the
        inputs, the analysis, the device-to-host read of the result."""
        if flush is not None:
            flush.zero_()
        ee[s_][0].record(stream)
        ensf.copy_sm(d_prior, h_prior, 152)
        d_y.copy_(h_y, non_blocking=True)
        if d_mask is not None:
            d_mask.copy_(h_mask, non_blocking=True)
        ei[s_][0].record(stream)
        analyse(d_prior, d_y, d_mask, 200 + s_)
        ei[s_][1].record(stream)
        ensf.copy_sm(h_out, out, 152)
        ee[s_][1].record(stream)
        # the host takes the result before the next analysis is enqueued
        torch.cuda.synchronize()

    # ---- timed region: K device-timed steps (inputs resident in HBM), the
    # first few each followed by one end-to-end step, so that both figures
    # are taken under the same conditions (a GB300 runs under its power cap
    # here; end-to-end steps taken after all the device steps, on a GPU that
    # had just run the test suite, came out 15-40 % slower than device step +
    # copies, while interleaved they differ by the copy time alone) ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for s_ in range(args.steps):
            if flush is not None:
                flush.zero_()
            ev[s_][0].record(stream)
            one(100 + s_)
            ev[s_][1].record(stream)
            if s_ < e2e_steps:
                e2e_step(s_)
        pipe = e2e_pipelined() if pipelined else None
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_each = [a.elapsed_time(b) for a, b in ev]
    ms = float(sum(step_each))
    if f.status_sync() != 0:
        raise RuntimeError("device error during the benchmark")
    e2e_each = [a.elapsed_time(b) for a, b in ee]
    seq = {"ms_per_step": [round(v, 2) for v in e2e_each],
           "h2d_ms": [round(ee[i][0].elapsed_time(ei[i][0]), 2) for i in range(e2e_steps)],
           "analysis_ms": [round(ei[i][0].elapsed_time(ei[i][1]), 2) for i in range(e2e_steps)],
           "d2h_ms": [round(ei[i][1].elapsed_time(ee[i][1]), 2) for i in range(e2e_steps)]}
    if pipelined:
        t0, t1, evs = pipe
        e2e_ms = t0.elapsed_time(t1) / pipe_steps
        e2e_parts = {"mode": f"{pipe_steps} analyses through host buffers, the copy-ins of the next ones and the "
                             f"copy-outs of the previous ones (two copy streams, three device sets) overlapping "
                             f"each analysis (Filter.analyses_from_host)",
                     "ms_per_step": round(e2e_ms, 2),
                     "copy_in_to_analysed_ms": [round(a.elapsed_time(b), 2) for a, b, _ in evs],
                     "analysed_to_copied_out_ms": [round(b.elapsed_time(c), 2) for _, b, c in evs],
                     "sequential_step": seq, "host_buffers": host_huge, "warm_copy_rounds_ms": warm}
    else:
        e2e_ms = float(sum(e2e_each)) / e2e_steps
        e2e_parts = dict(seq, mode="sequential: copy in, analyse, copy out, host takes the result",
                         host_buffers=host_huge, warm_copy_rounds_ms=warm)
    h2d = p.prior.nbytes + p.y.nbytes + (p.mask.nbytes if p.mask is not None else 0)
    d2h = p.n * p.d * 4
    # ---- per-kernel timing: the same steps again, every launch bracketed by
    # CUDA events on its stream (kept out of the timed region above, whose
    # small kernels the extra events would slow down) ----
    f.profile_enable(True)
    for s_ in range(args.steps):
        if flush is not None:
            flush.zero_()
        one(100 + s_)
    torch.cuda.synchronize()
    prof = f.profile_read()
    f.profile_enable(False)

    # ---- accuracy: one more analysis with the workload's own seed (and the
    # identity permutation for the mini-batch form), ensemble-mean RMSE
    # against the truth, beside the FP64 oracle's when the CPU baseline's
    # sample covers the whole analysis ----
    acc_out = torch.empty_like(prior)
    if J:
        f.analysis_minibatch(prior, y, mask, p.sigma_obs, p.K, p.eps,
                             torch.arange(p.n, dtype=torch.int32, device=dev), J, p.obs_op, seed=p.seed,
                             out=acc_out)
    else:
        f.analysis(prior, y, mask, p.sigma_obs, p.K, p.eps, p.obs_op, seed=p.seed, out=acc_out)
    truth_dev = torch.from_numpy(p.truth.astype(np.float32)).to(dev)
    _, gpu_rmse = ensf.ensemble_stats(acc_out, truth_dev)        # FP64 mean and RMSE (step a6)
    _, prior_rmse = ensf.ensemble_stats(prior, truth_dev)
    # the members themselves, for a per-member comparison with the oracle (small workloads)
    acc_members = acc_out.cpu().numpy() if p.n * p.d <= (64 << 20) else None
    # the big configuration: 64 members against the stored FP64 oracle rows
    # (tests/golden/make_large512_subsample.py; the oracle is exact on any
    # subset of members)
    subsample = None
    golden = os.path.join(ROOT, "tests", "golden", "large512_subsample64.npz")
    if rank == 0 and p.name == "large-512" and not J and os.path.exists(golden):  # rank 0 runs the stored seed
        g = np.load(golden)
        sub = acc_out[torch.from_numpy(g["rows"].astype(np.int64)).to(dev)].cpu().numpy().astype(np.float64)
        truth64 = p.truth.astype(np.float32).astype(np.float64)
        sub_rmse = float(np.sqrt(np.mean((sub.mean(axis=0) - truth64) ** 2)))
        ref_vals = g["values"]
        rel = np.linalg.norm(sub[:, g["idx"]] - ref_vals, axis=1) / np.linalg.norm(ref_vals, axis=1)
        # members whose oracle top-two log-kernel gap came within twice the
        # BF16 W X path's log-kernel error bound (they may follow another
        # forecast member than the oracle's)
        near = g["gap_ratio"] < 2.0 * 2.0 * 2.0 ** -9 / np.sqrt(p.d)
        subsample = {"members": int(len(g["rows"])), "gpu_rmse": sub_rmse, "oracle_rmse": float(g["rmse"]),
                     "rmse_rel_diff": abs(sub_rmse - float(g["rmse"])) / float(g["rmse"]),
                     "member_rel_err_on_sampled_entries": {"median": float(np.median(rel)),
                                                           "max": float(rel.max()), "entries": int(len(g["idx"])),
                                                           "max_away_from_ties": float(rel[~near].max())},
                     "near_tie_members": int(near.sum()),
                     "oracle": "FP64, %d host threads, %.0f s" % (int(g["threads"]), float(g["seconds"]))}
    del acc_out

    def _rmse(mean):
        return float(np.sqrt(np.mean((mean - p.truth.astype(np.float32).astype(np.float64)) ** 2)))
    accuracy = {"analysis_rmse": float(gpu_rmse.item()), "prior_rmse": float(prior_rmse.item()),
                "oracle_rmse": None}
    if subsample is not None:
        accuracy["oracle_subsample"] = subsample

    # ---- max over ranks ----
    ms, e2e_ms = max_over_ranks([ms, e2e_ms], dist, dev)
    if rank != 0:
        dist.destroy_process_group()
        return 0

    ms_per_step = ms / args.steps
    member_steps = p.n * p.K
    value = world * member_steps / (ms_per_step / 1e3)
    e2e_value = world * member_steps / (e2e_ms / 1e3)

    # ---- roofline of the dominant kernel (and of the other contraction) ----
    kernels = {k: v for k, v in prof.items() if v[1] > 0}
    peaks = _peaks()
    rooflines = {k: _roofline(k, kernels[k], p, gram, wx, args, peaks) for k in ("gram", "wx_em") if k in kernels}
    dom = max(kernels, key=lambda k: kernels[k][2])
    roof = rooflines.get(dom) or _roofline(dom, kernels[dom], p, gram, wx, args, peaks)
    other = {k: v for k, v in rooflines.items() if k != dom}
    # launches in the timed region: the profiled pass repeats the device-timed
    # analyses; the end-to-end analyses launch the same kernels
    per_analysis = sum(v[0] for v in prof.values()) / args.steps
    gpu_launches = int(round(per_analysis * (args.steps + e2e_steps + (pipe_steps if pipelined else 0))))

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step,
            "ms_each_step": {"median": float(np.median(step_each)), "min": float(min(step_each)),
                             "max": float(max(step_each))},
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"split-bf16": "bf16x3+bf16 (fp32 acc)", "split": "bf16x3 (fp32 acc)",
                                          "fp32": "f32", "tf32-bf16": "tf32+bf16 (fp32 acc)",
                                          "tf32": "tf32+bf16x3 (fp32 acc)",
                                          "bf16": "bf16 (fp32 acc)"}[args.path],
            "data": "synthetic", "config": dict(_config(p, args.path, world), minibatch_J=J or p.n),
            "roofline": roof, "accuracy": accuracy,
            "roofline_other": other,
            "kernels": {k: {"launches": v[0], "avg_ms": (v[2] / v[1]) if v[1] else None} for k, v in prof.items()},
            "e2e": dict({"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                        **e2e_parts),
            "gpu_launches": gpu_launches, "clocks": clk.summary(), "tuning": tuning, "cuda_graph": args.graph,
            "persistent": args.persistent}
    if not args.no_cpu_baseline:
        line["cpu_baseline"], oracle_out = cpu_baseline(p, args.cpu_budget_s, J or 0)
        if oracle_out is not None:
            accuracy["oracle_rmse"] = _rmse(oracle_out.mean(axis=0))
            if acc_members is not None:
                rel = np.linalg.norm(acc_members.astype(np.float64) - oracle_out, axis=1) / \
                    np.linalg.norm(oracle_out, axis=1)
                accuracy["member_rel_err"] = {"median": float(np.median(rel)), "p95": float(np.percentile(rel, 95)),
                                              "max": float(rel.max())}
            accuracy["rmse_rel_diff"] = abs(accuracy["analysis_rmse"] / accuracy["oracle_rmse"] - 1.0)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def run_sharded(args):
    """One filter whose state is split along d over the ranks, one per GPU
    (the paper's single large-state EnSF on many GPUs, Sec. IV-B): every rank
    runs the per-slice kernels on its columns; the split-K partial Grams are
    all-gathered over NCCL every Euler-Maruyama step and the FP64 norms
    all-reduced once per analysis (paper_2407_12168_gb300.sharded).  Strong
    scaling: the same filter whatever the number of ranks."""
    import types

    import torch
    import torch.distributed as dist
    rank, local_rank, world = _dist_env()
    torch.cuda.set_device(local_rank)
    dist.init_process_group("nccl")
    from paper_2407_12168_gb300 import ensf, sharded

    gram, wx = PATHS[args.path]
    p = make_problem(args.workload, 0)               # one filter, the same on every rank
    c0, dl = sharded.split_columns(p.d, world)[rank]
    dev = torch.device("cuda", local_rank)
    prior = torch.from_numpy(np.ascontiguousarray(p.prior[:, c0:c0 + dl])).to(dev)
    y = torch.from_numpy(np.ascontiguousarray(p.y[c0:c0 + dl])).to(dev)
    mask = None if p.mask is None else torch.from_numpy(np.ascontiguousarray(p.mask[c0:c0 + dl])).to(dev)
    out = torch.empty_like(prior)
    be = sharded.CudaShardBackend(p.n, dl, gram=gram, wx=wx, inline_noise=args.inline_noise)
    # launch shapes: rank 0 tunes on its slice, every rank records the same
    # shapes (the split count fixes the layout of the gathered partials)
    tuning = None
    if gram != "fp32" or wx != "fp32":
        if args.set_tuning:
            tuning = dict(json.loads(args.set_tuning))
        elif rank == 0:
            tuning = be.f.autotune(prior, y, mask, p.sigma_obs, p.eps, p.obs_op, seed=p.seed, out=out)
        box = [tuning]
        dist.broadcast_object_list(box, src=0)
        tuning = box[0]
        keep = ("gram_tile_n", "gram_stages", "gram_k_block", "gram_splits", "wx_tile_n", "gram_cta_pair",
                "gram_noise_warps", "gram_fp32_particles", "noise_inline", "pdl")
        be.f.set_tuning(p.n, dl, **{k: v for k, v in tuning.items() if k in keep})
    args.tuning = tuning
    try:
        store = dist.distributed_c10d._get_default_store()
    except Exception:
        store = None
    ex = sharded.TorchExchange(store=store, heartbeat_timeout_s=120.0)
    run = sharded.ShardedAnalysis(be, ex)
    S_all = [None] * world
    dist.all_gather_object(S_all, run.S)
    if len(set(S_all)) != 1:
        raise RuntimeError(f"ranks disagree on the split count: {S_all}")
    stream = torch.cuda.current_stream()

    def analyse(pr, yy, mm, k_seed):
        return run.run(pr, yy, mm, p.sigma_obs, p.K, p.eps, c0, obs_op=p.obs_op, seed=p.seed + k_seed, out=out)

    for w in range(args.warmup):
        analyse(prior, y, mask, w)
    torch.cuda.synchronize()
    # end-to-end: this rank's slice copied in from page-locked host memory and its result copied out
    sl = types.SimpleNamespace(prior=np.ascontiguousarray(p.prior[:, c0:c0 + dl]),
                               y=np.ascontiguousarray(p.y[c0:c0 + dl]),
                               mask=None if p.mask is None else np.ascontiguousarray(p.mask[c0:c0 + dl]))
    h_prior, h_y, h_mask, h_out, host_huge = _host_buffers(ensf, sl, args.small_pages, args.any_node)
    d_prior, d_y = torch.empty_like(prior), torch.empty_like(y)
    d_mask = torch.empty_like(mask) if mask is not None else None
    e2e_steps = max(1, min(args.steps, 3))
    ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

    def e2e_step(s_):
        ee[s_][0].record(stream)
        ensf.copy_sm(d_prior, h_prior, 152)
        d_y.copy_(h_y, non_blocking=True)
        if d_mask is not None:
            d_mask.copy_(h_mask, non_blocking=True)
        res = analyse(d_prior, d_y, d_mask, 200 + s_)
        ensf.copy_sm(h_out, res, 152)
        ee[s_][1].record(stream)
        torch.cuda.synchronize()

    warm = _warm_host_copies(ensf, stream, [(d_prior, h_prior), (h_out, d_prior)],
                             [(h_out, d_prior), (d_prior, h_prior)])
    host_huge["warm_copy_rounds_ms"] = warm
    dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for s_ in range(args.steps):
            ev[s_][0].record(stream)
            analyse(prior, y, mask, 100 + s_)
            ev[s_][1].record(stream)
            if s_ < e2e_steps:
                e2e_step(s_)
        torch.cuda.synchronize()
    dist.barrier()
    step_each = [a.elapsed_time(b) for a, b in ev]
    ms = float(sum(step_each))
    e2e_ms = float(sum(a.elapsed_time(b) for a, b in ee)) / e2e_steps
    if be.f.status_sync() != 0:
        raise RuntimeError("device error during the benchmark")
    be.f.profile_enable(True)
    for s_ in range(args.steps):
        analyse(prior, y, mask, 100 + s_)
    torch.cuda.synchronize()
    prof = be.f.profile_read()
    be.f.profile_enable(False)
    # accuracy: ensemble-mean RMSE over all columns, from every slice's squared errors
    acc = analyse(prior, y, mask, 0).clone()
    truth_dev = torch.from_numpy(np.ascontiguousarray(p.truth[c0:c0 + dl]).astype(np.float32)).to(dev)
    _, rmse_slice = ensf.ensemble_stats(acc, truth_dev)
    sq = torch.tensor([float(rmse_slice.item()) ** 2 * dl], dtype=torch.float64, device=dev)
    dist.all_reduce(sq)
    # the stored FP64 oracle rows of the large workload: each rank contributes its columns
    golden = os.path.join(ROOT, "tests", "golden", "large512_subsample64.npz")
    sub_parts = None
    if p.name == "large-512" and os.path.exists(golden):
        g = np.load(golden)
        idx = g["idx"]
        mine = (idx >= c0) & (idx < c0 + dl)
        rows = torch.from_numpy(g["rows"].astype(np.int64)).to(dev)
        vals = acc[rows][:, torch.from_numpy(idx[mine] - c0).to(dev)].cpu().numpy().astype(np.float64)
        sub_parts = [None] * world
        dist.all_gather_object(sub_parts, (np.flatnonzero(mine), vals))
    ms, e2e_ms = max_over_ranks([ms, e2e_ms], dist, dev)
    if rank != 0:
        dist.destroy_process_group()
        return 0
    ms_per_step = ms / args.steps
    member_steps = p.n * p.K
    accuracy = {"analysis_rmse": float(np.sqrt(sq.item() / p.d))}
    if sub_parts is not None:
        vals = np.zeros((len(g["rows"]), len(g["idx"])))
        for pos, v in sub_parts:
            vals[:, pos] = v
        ref_vals = g["values"]
        rel = np.linalg.norm(vals - ref_vals, axis=1) / np.linalg.norm(ref_vals, axis=1)
        accuracy["oracle_subsample"] = {"members": int(len(g["rows"])), "entries": int(len(g["idx"])),
                                        "member_rel_err": {"median": float(np.median(rel)),
                                                           "max": float(rel.max())}}
    kernels = {k: v for k, v in prof.items() if v[1] > 0}
    peaks = _peaks()
    pl = types.SimpleNamespace(n=p.n, d=dl, name=p.name + f"-slice{world}")
    rooflines = {k: _roofline(k, kernels[k], pl, gram, wx, args, peaks) for k in ("gram", "wx_em") if k in kernels}
    for r_ in rooflines.values():
        r_["traffic"] = None  # no capture of the per-slice shapes
    dom = max(kernels, key=lambda k: kernels[k][2])
    line = {"metric": METRIC, "value": member_steps / (ms_per_step / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "ms_each_step": {"median": float(np.median(step_each)), "min": float(min(step_each)),
                             "max": float(max(step_each))},
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": {"split-bf16": "bf16x3+bf16 (fp32 acc)", "split": "bf16x3 (fp32 acc)",
                      "fp32": "f32"}.get(args.path, args.path),
            "data": "synthetic",
            "config": dict(_config(p, args.path, world),
                           parallelism=f"one filter, d split over {world} GPUs ({dl} columns each), "
                                       f"Gram partials all-gathered over NCCL per step"),
            "roofline": rooflines.get(dom) or _roofline(dom, kernels[dom], pl, gram, wx, args, peaks),
            "roofline_other": {k: v for k, v in rooflines.items() if k != dom},
            "accuracy": accuracy,
            "kernels": {k: {"launches": v[0], "avg_ms": (v[2] / v[1]) if v[1] else None} for k, v in prof.items()},
            "e2e": {"value": member_steps / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": p.prior.nbytes + p.y.nbytes + (p.mask.nbytes if p.mask is not None else 0),
                    "d2h_bytes_per_step": p.n * p.d * 4, "host_buffers": host_huge},
            "gpu_launches": int(sum(v[0] for v in prof.values())) * world,
            "clocks": clk.summary(), "tuning": tuning, "split_k_per_rank": run.S}
    if not args.no_cpu_baseline:
        line["cpu_baseline"], _ = cpu_baseline(p, args.cpu_budget_s)
    print(json.dumps(line))
    dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="large-512", choices=sorted(inputs.WORKLOADS) + ["batched-uneven"])
    ap.add_argument("--path", default="split-bf16", choices=sorted(PATHS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--graph", action="store_true", help="replay each analysis as one captured CUDA graph")
    ap.add_argument("--inline-noise", action="store_true",
                    help="tensor-core W X evaluates the noise in its epilogue (no pre-generated slice)")
    ap.add_argument("--set-tuning", default=None, metavar="JSON",
                    help='launch shapes instead of the autotuner, e.g. {"gram_tile_n": 256, "gram_stages": 3, '
                         '"gram_splits": 4, "gram_cta_pair": 1, "wx_tile_n": 256}')
    ap.add_argument("--persistent", action="store_true",
                    help="fp32 path, N <= 128: all K steps in one cooperative launch")
    ap.add_argument("--minibatch", type=int, default=0, metavar="J",
                    help="mini-batch prior score over J members per Euler-Maruyama step (tensor-core paths)")
    ap.add_argument("--replicas", action="store_true",
                    help="with several GPUs: one independent filter per GPU (weak scaling) instead of one "
                         "filter split along d over the GPUs")
    ap.add_argument("--sharded", action="store_true",
                    help="the d-sharded mode also on one GPU (under torchrun: exercises the NCCL exchange)")
    ap.add_argument("--any-node", action="store_true",
                    help="host buffers without the preference for the device's nearest NUMA node (comparison)")
    ap.add_argument("--small-pages", action="store_true",
                    help="end-to-end host buffers pinned without huge pages (for comparison)")
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--ref-step-s", type=float, default=8.0)
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        print("note: warm-up raised to the minimum of 3", file=sys.stderr)
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched-uneven":
        return run_batched(args)
    if (_dist_env()[2] > 1 and not args.replicas) or args.sharded:
        # the communicator's rank count appears in NCCL's own init lines
        os.environ.setdefault("NCCL_DEBUG", "INFO")
        os.environ.setdefault("NCCL_DEBUG_SUBSYS", "INIT")
        return run_sharded(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
