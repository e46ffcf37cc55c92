"""Benchmark: K-NNG build time by NN-Descent on one GB300 (and N replicas).

Headline workload: 1,000,000 points in 128 dimensions from an equal-weight
mixture of 1,000 Gaussian clusters (centres N(0, 4 I), sigma 0.5), K = 32,
float32.  Its stated parameters (rho 0.3, delta 0.001, 12 iterations) stop at
recall@K 0.964, below the metric's 0.99, and more iterations do not raise it:
the timed build runs the recall-0.99 operating point of a measured ladder
(rho 0.7, the other parameters as stated), named in config.workload; the
stated point, the bf16 form and the ladder are reported beside it.

A step is one whole build (random init, every iteration that runs, re-ranked
output) with the points already resident on the device.  The L2 cache is
flushed (a 256 MiB device write) between timed steps, outside the timed
region.  With --gpus N (torchrun) every rank builds its own replica: the path
has no exchange step, so the ranks share nothing but the barrier and the
max-over-ranks of the step time.

Printed (rank 0, one JSON line): the build time, recall@K on 10,000 sampled
rows against the GPU brute force (NN-Descent seeds 0, 1, 2), distance
evaluations per second, the end-to-end time through the public API with host
buffers, the roofline of the dominant kernel (the local join), and the CPU
oracle timed on this host on a bounded sample of the workload.

--impl reference times the CPU oracle on a bounded sample of the same
workload instead: the reference arm.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

WORKLOAD = "mixture_n1m_d128"
METRIC = "K-NNG build s at recall@K>=0.99"
RECALL_ROWS = 2000

# Recall-0.99 operating points (rho, delta, max_iters) of workloads whose
# stated parameters stop short of recall 0.99, from measured ladders: the
# smallest sample rate that reaches 0.99 on every one of NN-Descent seeds 0-2,
# the other parameters as stated (1M x 128: rho 0.5 / 0.6 / 0.7 gave 0.984 /
# 0.989 / 0.991, and a smaller delta or a larger cap changed nothing; 100k x
# 16: rho 0.55 gave 0.9906)
RECALL99 = {
    "mixture_n1m_d128": (0.7, 0.001, 12),
    "clustered_n100k_d16": (0.55, 0.001, 15),
    "mnist_like_n70k_d784": (0.6, 0.001, 15),
    "audio_like_n54k_d192": (0.7, 0.001, 15),
}
# ladders reported beside the timed point: (rho, delta, max_iters)
LADDER = {
    "mixture_n1m_d128": [(0.3, 0.001, 12), (0.3, 0.0, 30), (0.5, 0.001, 12), (0.6, 0.001, 12),
                         (0.7, 0.001, 12), (1.0, 0.001, 12)],
    "clustered_n100k_d16": [(0.5, 0.001, 15), (0.55, 0.001, 15), (0.6, 0.001, 15)],
    "mnist_like_n70k_d784": [(0.5, 0.001, 15), (0.6, 0.001, 15), (0.7, 0.001, 15), (1.0, 0.001, 15)],
    "audio_like_n54k_d192": [(0.5, 0.001, 15), (0.6, 0.001, 15), (0.7, 0.001, 15), (0.8, 0.001, 15)],
}
GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_recall.json")


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class _Nvml:
    """Minimal in-process NVML reader (ctypes): SM clock, max SM clock and the
    clock-event reasons, without spawning a process per sample."""

    HW_SLOWDOWN, SW_POWER_CAP = 0x8, 0x4
    HW_THERMAL, SW_THERMAL = 0x40, 0x20

    def __init__(self, index: int):
        import ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        self.c = ctypes
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(index, ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle")

    def sample(self):
        c = self.c
        sm, mx, reasons = c.c_uint(), c.c_uint(), c.c_ulonglong()
        self.lib.nvmlDeviceGetClockInfo(self.h, 1, c.byref(sm))            # NVML_CLOCK_SM
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, c.byref(mx))
        self.lib.nvmlDeviceGetCurrentClocksEventReasons(self.h, c.byref(reasons))
        r = reasons.value
        names = [nm for nm, bit in (("hw_slowdown", self.HW_SLOWDOWN), ("hw_thermal_slowdown", self.HW_THERMAL),
                                    ("sw_thermal_slowdown", self.SW_THERMAL), ("sw_power_cap", self.SW_POWER_CAP))
                 if r & bit]
        return float(sm.value), float(mx.value), names


class ClockSampler:
    """SM clocks and throttle reasons sampled during the timed region: NVML in
    process every 10 ms (nvidia-smi every 200 ms if NVML cannot be loaded)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []  # (sm_mhz, max_mhz, [reasons])
        self._stop = threading.Event()
        self._t = None
        try:
            self.nvml = _Nvml(index)
        except Exception:
            self.nvml = None

    def _smi(self):
        out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=5).stdout.strip()
        r = [c.strip() for c in out.split(",")]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        return (float(r[1]), float(r[2]), [nm for nm, v in zip(names, r[5:9]) if v.lower() == "active"])

    def _run(self):
        while not self._stop.is_set():
            try:
                self.samples.append(self.nvml.sample() if self.nvml else self._smi())
            except Exception:
                pass
            self._stop.wait(0.01 if self.nvml else 0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        sm = [x[0] for x in self.samples]
        mx = [x[1] for x in self.samples]
        reasons = sorted({r for x in self.samples for r in x[2]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples),
                "source": "nvml" if self.nvml else "nvidia-smi"}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(v: float, ws: int, device):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def join_bytes(st: dict, dp: int) -> float:
    """Algorithmic bytes of the local-join launches of one build: every
    candidate id read (4 B), every gathered candidate row (dp * 4 B) with its
    worst-key snapshot (8 B), every proposal key written (8 B)."""
    return st["cand_ids"] * 4.0 + st["gathered_rows"] * (dp * 4.0 + 8.0) + st["proposals"] * 8.0


def merge_bytes(st: dict) -> float:
    """Algorithmic bytes of the list-merge launches of one build: every
    proposal key read (8 B), and per merged list one K-key list read and
    written (2 * K * 8 B)."""
    return st["proposals"] * 8.0 + st["merges"] * 2.0 * st["K"] * 8.0


def measured_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu record in
    profiles/traffic.json, or None when the kernel's sources changed since the
    capture (their sha256 no longer matches) or no record exists."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        h = hashlib.sha256()
        for p in rec["sources"]:
            h.update(open(os.path.join(ROOT, p), "rb").read())
        if h.hexdigest() != rec["sources_sha256"]:
            return None
        return rec["dram_bytes_per_launch"]
    except Exception:
        return None


def deal_by_cost(costs, ranks: int):
    """Data sets dealt over ranks by their cost (n * d, the work of a build
    grows with both): largest first, each to the rank with the least load so
    far (longest-processing-time rule; the heaviest rank carries at most the
    mean load plus one data set's cost).  Returns, per rank, its data-set
    indices in ascending order."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * ranks
    out = [[] for _ in range(ranks)]
    for i in order:
        r = min(range(ranks), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(x) for x in out]


def run_batched(args):
    """256 independent data sets: one batched build (one launch per step for
    all data sets of a row-width class) against 256 sequential float32
    builds.  With N ranks the data sets are dealt out by cost, n * d (no
    collective: they are independent), and the step time is the slowest
    rank's."""
    import torch

    import paper_2112_06630_gb300 as knng
    from oracle import metrics

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    cfg = workloads.BATCHED
    all_sets = workloads.batched_data(cfg["count"], cfg["seed"])
    mine = deal_by_cost([x.shape[0] * x.shape[1] for x in all_sets], ws)[rank]
    sets = [all_sets[i] for i in mine]
    xs = [torch.from_numpy(x).to(device) for x in sets]
    # the batched form as built: each width class's loop one captured graph,
    # its join kernel and block shape picked by the autotuner (--batched-plain
    # switches both off)
    tuned = not args.batched_plain
    flags = (knng.FLAG_BF16 if args.bf16 else 0) | (knng.FLAG_GRAPH if (args.graph or tuned) else 0) | \
        (knng.FLAG_AUTOTUNE if (args.autotune or tuned) else 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    K, rho, delta, it = cfg["K"], cfg["rho"], cfg["delta"], cfg["max_iters"]

    def timed(fn):
        flush.fill_(1)
        _barrier(ws)
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        out = fn()
        e.record()
        torch.cuda.synchronize()
        return s.elapsed_time(e) / 1e3, out

    batched = lambda: knng.knng_build_batched(xs, K, rho, delta, it, seed=0, flags=flags)
    sequential = lambda: [knng.knng_build(x, K, rho, delta, it, seed=0) for x in xs]
    for _ in range(args.warmup):
        batched()
    tb, tsq = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            t, (outs, st) = timed(batched)
            tb.append(t)
    for _ in range(max(1, min(args.steps, 3))):
        t, seq = timed(sequential)
        tsq.append(t)
    # end to end through the public API: pinned host inputs, host outputs
    xh = [torch.from_numpy(x).pin_memory() for x in sets]
    te = []
    for i in range(args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        knng.knng_build_batched(xh, K, rho, delta, it, seed=0, flags=flags)
        t1 = time.perf_counter()
        if i >= args.warmup:
            te.append(t1 - t0)
    vb = _max_over_ranks(sum(tb) / len(tb), ws, device)
    vs = _max_over_ranks(sum(tsq) / len(tsq), ws, device)
    ve = _max_over_ranks(sum(te) / len(te), ws, device)
    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    g = np.random.default_rng(1)
    hits, tot = 0.0, 0
    for b in g.choice(len(sets), 8, replace=False):
        rows = g.choice(len(sets[b]), min(250, len(sets[b])), replace=False)
        bi, _ = knng.knng_bruteforce(xs[b], K, rows=torch.from_numpy(rows).to(device))
        r = metrics.recall(sets[b], outs[b][0].cpu().numpy(), bi.cpu().numpy(), rows)
        hits += r * len(rows)
        tot += len(rows)
    line = {
        "metric": METRIC, "value": round(vb, 6), "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(vb * 1e3, 3), "higher_is_better": False,
        "scaling": "strong" if ws > 1 else "weak",
        "vs_baseline": None, "dtype": "bf16+f32" if args.bf16 else "f32", "data": "synthetic",
        "config": {"workload": "batched_256", "datasets": len(all_sets),
                   "total_n": int(sum(len(x) for x in all_sets)), "K": K, "rho": rho, "delta": delta,
                   "max_iters": it, "bf16": bool(args.bf16), "graph": bool(args.graph or tuned),
                   "autotune": bool(args.autotune or tuned),
                   "parallelism": f"data sets dealt over {ws} rank(s) by n*d (largest first, least-loaded rank)",
                   "l2": "flushed between timed steps (256 MiB write)", "inputs": "device-resident"},
        "e2e": {"value": round(ve, 6), "unit": "s", "h2d_bytes_per_step": int(sum(x.nbytes for x in sets)),
                "d2h_bytes_per_step": int(sum(len(x) for x in sets) * K * 8)},
        "sequential_fp32_s": round(vs, 4), "speedup_vs_sequential": round(vs / vb, 2),
        "recall_at_k": round(hits / tot, 5), "recall_rows": tot, "dist_evals": st["dist_evals"],
        "recall_0.99": {"reached": hits / tot >= 0.99,
                        "note": "no sample rate takes this workload to 0.99 at K = 16: measured 0.955 (rho 0.5) "
                                "to 0.985 (rho 1.0), converged; its hardest set stops near 0.71 and the oracle's "
                                "build of it at 0.70, so the ceiling is the method's"},
        "gpu_launches": int(st["kernel_launches"]), "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_sweep(args):
    """Dimension sweep (the paper's d = 8 ... 3144 in steps of 64 at n =
    16,384 on the Single Gaussian set, covariance 2 I; K = 20, rho = 0.5,
    delta = 0.001, at most 15 iterations), float32 and bf16, then the two
    roofline placements at n = 131,072, d in {8, 256}.  One JSON line per
    run: build time, local-join time per launch, distance evaluations per
    second, the paper's flop rate (evals * (3d - 1) / s) and the join's
    achieved bytes per second."""
    import torch

    import paper_2112_06630_gb300 as knng

    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    K, rho, delta, it = 20, 0.5, 0.001, 15
    runs = [(16384, d) for d in range(8, 3145, 64)] + [(131072, 8), (131072, 256)]
    for n, d in runs:
        x = torch.from_numpy(workloads.single_gaussian(n, d, seed=d, var=2.0)).to(device)
        for bf16 in (False, True):
            if bf16 and d < 64:
                continue
            flags = knng.FLAG_BF16 if bf16 else 0
            for _ in range(2):
                knng.knng_build(x, K, rho, delta, it, seed=0, flags=flags)
            ts = []
            for _ in range(3):
                flush.fill_(1)
                torch.cuda.synchronize()
                s0 = torch.cuda.Event(enable_timing=True)
                e0 = torch.cuda.Event(enable_timing=True)
                s0.record()
                _, _, st = knng.knng_build(x, K, rho, delta, it, seed=0, flags=flags)
                e0.record()
                torch.cuda.synchronize()
                ts.append(s0.elapsed_time(e0) / 1e3)
            _, _, tst = knng.knng_build(x, K, rho, delta, it, seed=0, flags=flags | knng.FLAG_TIMING)
            t = sum(ts) / len(ts)
            ran = max(1, tst["join_ran"])
            dp = (d + 63) // 64 * 32 if bf16 and d >= 64 else (d + 3) // 4 * 4
            jt = tst["join_ms_ran"] / 1e3 / ran
            print(json.dumps({"sweep": "dimension", "n": n, "d": d, "bf16": bf16, "build_s": round(t, 6),
                              "iterations": st["iterations"], "join_path": st["join_path"],
                              "join_ms_per_launch": round(jt * 1e3, 4),
                              "dist_evals_per_s": round(st["dist_evals"] / t, 1),
                              "paper_flops_per_s": round(st["dist_evals"] * (3 * d - 1) / t, 1),
                              "join_gb_per_s": round(join_bytes(tst, dp) / ran / jt / 1e9, 1)}), flush=True)


def run_bruteforce(args):
    """Exact K-NNG by brute force (Section 2 definition; the ground truth) on
    the workload's points: all rows, or --rows R sampled query rows.  One JSON
    line: seconds per call with device-resident input, the end-to-end call
    from pinned host memory, the pair rate, the roofline of the tensor-core
    prefilter (its bf16 MMA work: three products of 2 * dpb flops for each
    padded query-point pair, against the measured cuBLAS bf16 peak) and the
    oracle on a bounded sample of queries."""
    import numpy as np
    import torch

    import oracle
    import paper_2112_06630_gb300 as knng

    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    w, x, wname = _workload(args)
    n, d, K = x.shape[0], x.shape[1], w.K
    nq = n if not args.rows else min(args.rows, n)
    rows_h = None if nq == n else np.sort(np.random.default_rng(0).choice(n, nq, replace=False)).astype(np.int64)
    xd = torch.from_numpy(x).to(device)
    rows_d = None if rows_h is None else torch.from_numpy(rows_h).to(device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    for _ in range(args.warmup):
        knng.knng_bruteforce(xd, K, rows=rows_d)
    torch.cuda.synchronize()
    ts, pf, fb = [], [], []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            s0 = torch.cuda.Event(enable_timing=True)
            e0 = torch.cuda.Event(enable_timing=True)
            s0.record()
            knng.knng_bruteforce(xd, K, rows=rows_d)
            e0.record()
            torch.cuda.synchronize()
            ts.append(s0.elapsed_time(e0) / 1e3)
            pf.append(knng.bruteforce_last_prefilter_ms())
            fb.append(knng.bruteforce_last_fallbacks())
    step_s = sum(ts) / len(ts)
    # end to end: pinned host input and query ids, host outputs
    xh = torch.from_numpy(x).pin_memory()
    e2e = []
    for i in range(args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        knng.knng_bruteforce(xh, K, rows=rows_h)
        e2e.append(time.perf_counter() - t0)
    e2e_s = sum(e2e[args.warmup:]) / args.steps
    tensor = pf[0] >= 0
    roof = None
    if tensor:
        peaks = _peaks()
        peak = peaks["bf16_tflops"] if peaks else 1900.0
        dpb = ((d + 3) // 4 * 4 + 15) // 16 * 16
        pad = lambda v: (v + 127) // 128 * 128
        flops = 3.0 * 2.0 * dpb * pad(nq) * pad(n)
        pms = sum(pf) / len(pf) / 1e3
        ach = flops / pms / 1e12
        roof = {"kernel": "bf_tc_kernel", "bound": "tensor", "achieved": round(ach, 1), "peak": peak,
                "unit": "TFLOP/s", "frac": round(ach / peak, 4), "traffic": None,
                "peak_source": "measured bf16 burst" if peaks else "fallback",
                "flops_per_launch": flops, "launch_ms": round(pms * 1e3, 4),
                "share_of_call": round(pms / step_s, 3)}
    cpu = None
    if not args.no_cpu:
        # the oracle on a bounded sample of queries, scaled to the whole call
        g = np.random.default_rng(1)
        sample, spent, t0 = 0, 0.0, time.perf_counter()
        while spent < 10.0 and sample < nq:
            q = int(g.integers(0, n)) if rows_h is None else int(rows_h[g.integers(0, nq)])
            oracle.bruteforce(x, K, rows=np.array([q], dtype=np.int64))
            sample += 1
            spent = time.perf_counter() - t0
        cpu = {"value": round(spent / sample * nq, 3), "unit": "s", "cores": 1, "kind": "oracle",
               "sample": f"{sample} query rows against all {n} points, scaled to {nq} queries"}
    launches = (7 + (3 if max(fb) > 0 else 0)) if tensor else 3
    line = {
        "metric": "exact K-NNG rows by brute force, s per call", "value": round(step_s, 6), "unit": "s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 prefilter + f32" if tensor else "f32", "data": "synthetic",
        "config": {"workload": wname, "n": n, "d": d, "K": K, "queries": nq,
                   "path": "tensor cores" if tensor else "CUDA cores",
                   "l2": "flushed between timed steps (256 MiB write)", "inputs": "device-resident"},
        "pairs_per_s": round(nq * (n - 1) / step_s, 1),
        "uncertified_queries": fb[-1],
        "e2e": {"value": round(e2e_s, 6), "unit": "s", "h2d_bytes_per_step": int(x.nbytes) + (0 if rows_h is None
                else int(rows_h.nbytes)), "d2h_bytes_per_step": int(nq * K * 8)},
        "gpu_launches": launches * args.steps,
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_relabel_ab(args):
    """Relabelling after iteration 1 (Section 3.2): none, Algorithm 1 (exact,
    sequential) and the parallel single-linkage variant.  One JSON line per
    workload and variant: build time (CUDA events, L2 flushed), the
    relabelling's own time (events around it), local-join time per running
    iteration, recall on 2,000 sampled rows, and the window purity of the
    layout -- the Fig. 4 measure: the fraction of the most frequent cluster
    in each window of 2,000 spots."""
    import numpy as np
    import torch

    import paper_2112_06630_gb300 as knng
    from oracle import metrics

    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    cases = [
        # name, n, d, K, rho, delta, iterations, mixture parameters (Fig. 4: 8 clusters)
        ("clustered_n16k_d8_c8", 16384, 8, 20, 0.5, 0.001, 15, dict(clusters=8)),
        ("clustered_n100k_d16", 100_000, 16, 20, 0.5, 0.001, 15, dict(clusters=50)),
        ("mixture_n1m_d128", 1_000_000, 128, 32, 0.3, 0.001, 12, dict(clusters=1000, centre_std=2.0, sigma=0.5)),
    ]
    variants = [("none", 0), ("algorithm1", knng.FLAG_REORDER),
                ("parallel", knng.FLAG_REORDER | knng.FLAG_REORDER_PARALLEL),
                ("parallel_again_after_4", knng.FLAG_REORDER | knng.FLAG_REORDER_PARALLEL)]

    def build_again(xd, K, rho, delta, iters, flags, timing=0):
        # relabel after iteration 1 (automatic) and again after iteration 4,
        # through the step API
        c = knng.Context(xd, K, rho=rho, delta=delta, seed=0, flags=flags | timing)
        done = False
        for it in range(min(4, iters)):
            done = c.iterate()[0]
            if done:
                break
        if not done and iters > 4:
            c.reorder()
            c.run(iters - 4)
        return c
    for name, n, d, K, rho, delta, iters, mp in cases:
        x, lab = workloads.gaussian_mixture(n, d, seed=0, return_labels=True, **mp)
        xd = torch.from_numpy(x).to(device)
        rows = np.random.default_rng(0).choice(n, RECALL_ROWS, replace=False)
        ei, _ = knng.knng_bruteforce(xd, K, rows=torch.from_numpy(rows).to(device))
        ei = ei.cpu().numpy()
        nclu = int(lab.max()) + 1
        for vname, flags in variants:
            steps = args.steps if not (vname == "algorithm1" and n > 200_000) else min(args.steps, 2)
            for _ in range(min(args.warmup, 2) if steps < args.steps else args.warmup):
                knng.knng_build(xd, K, rho, delta, iters, seed=0, flags=flags)
            again = vname == "parallel_again_after_4"
            ts = []
            for _ in range(steps):
                flush.fill_(1)
                torch.cuda.synchronize()
                s0 = torch.cuda.Event(enable_timing=True)
                e0 = torch.cuda.Event(enable_timing=True)
                if again:
                    t0 = time.perf_counter()
                    c = build_again(xd, K, rho, delta, iters, flags)
                    gi_d, _ = c.get(device=True)
                    torch.cuda.synchronize()
                    ts.append(time.perf_counter() - t0)  # host clock: the step API synchronises
                    c.close()
                    continue
                s0.record()
                knng.knng_build(xd, K, rho, delta, iters, seed=0, flags=flags)
                e0.record()
                torch.cuda.synchronize()
                ts.append(s0.elapsed_time(e0) / 1e3)
            if again:
                c = build_again(xd, K, rho, delta, iters, flags, knng.FLAG_TIMING)
            else:
                c = knng.Context(xd, K, rho=rho, delta=delta, seed=0, flags=flags | knng.FLAG_TIMING)
                c.run(iters)
            with c:
                st = c.stats()
                sg = c.permutation()
                gi, _ = c.get(device=False)
            inv = np.empty(n, np.int64)
            inv[sg] = np.arange(n)
            pur = metrics.window_purity(lab[inv], 2000, nclu)
            ran = max(1, st["join_ran"])
            print(json.dumps({
                "relabel": vname, "workload": name, "n": n, "d": d, "K": K, "clusters": nclu,
                "build_s": round(sum(ts) / len(ts), 6), "steps": steps,
                "relabel_ms": round(st["reorder_ms"], 3), "iterations": st["iterations"],
                "join_ms_per_iter": round(st["join_ms_ran"] / ran, 4),
                "recall_at_k": round(metrics.recall(x, gi, ei, rows), 5),
                "window_purity": {"windows": len(pur), "mean": round(float(pur.mean()), 4),
                                  "min": round(float(pur.min()), 4), "last": round(float(pur[-1]), 4)},
            }), flush=True)


def _op_point(args):
    """(workload with overrides, data, name, timed point): the timed point is
    the workload's recall-0.99 operating point when no override is given and
    the stated parameters stop short of 0.99, else the (overridden) workload."""
    import dataclasses
    w, x, wname = _workload(args)
    overridden = any(v is not None for v in (args.n, args.rho, args.delta, args.max_iters))
    if not overridden and args.workload in RECALL99:
        rho, delta, iters = RECALL99[args.workload]
        op = dataclasses.replace(w, rho=rho, delta=delta, max_iters=iters)
        wname = f"{args.workload}_rho{rho}_delta{delta}_iters{iters}"
    else:
        op = w
    return w, x, wname, op, overridden


def _time_builds(knng, xd, op, flags, steps, warmup, flush, stream, ws=1, seed=0):
    """Mean CUDA-event time of `steps` whole builds after `warmup` untimed ones
    (L2 flushed before each timed build, barrier and synchronisation on both
    sides), and the last build's outputs."""
    import torch
    for _ in range(warmup):
        knng.knng_build(xd, op.K, op.rho, op.delta, op.max_iters, seed=seed, flags=flags)
    times, out = [], None
    for _ in range(steps):
        flush.fill_(1)
        _barrier(ws)
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        out = knng.knng_build(xd, op.K, op.rho, op.delta, op.max_iters, seed=seed, flags=flags)
        e.record(stream)
        torch.cuda.synchronize()
        _barrier(ws)
        times.append(s.elapsed_time(e) / 1e3)
    return sum(times) / len(times), out


JOIN_KERNELS = {0: "join_kernel", 1: "tile_join_kernel", 2: "set_kernel+ring_join_kernel",
                3: "set_kernel+pipe_join_kernel", 4: "set_kernel+pipe_join_kernel<8,2>"}


def run_gpu(args):
    import dataclasses

    import torch

    import paper_2112_06630_gb300 as knng
    from oracle import metrics

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)

    w, x, wname, op, overridden = _op_point(args)
    xd = torch.from_numpy(x).to(device)
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    flags = (knng.FLAG_REORDER if args.reorder else 0) | (knng.FLAG_BF16 if args.bf16 else 0) | \
        (knng.FLAG_GRAPH if args.graph else 0) | (knng.FLAG_AUTOTUNE if args.autotune else 0) | \
        (knng.FLAG_HEAP_SAMPLING if args.heap else 0) | (knng.FLAG_FP8 if args.fp8 else 0) | \
        (knng.FLAG_REORDER | knng.FLAG_REORDER_PARALLEL if args.reorder_parallel else 0)
    # float32 words per gathered row (bf16 rows: 2 bytes an element, e4m3: 1)
    if args.fp8 and w.d >= 64:
        dp = (w.d + 63) // 64 * 64 // 4
    elif args.bf16 and w.d >= 64:
        dp = (w.d + 63) // 64 * 64 // 2
    else:
        dp = (w.d + 3) // 4 * 4

    with ClockSampler(local) as clk:
        step_s, (ids, dists, stats) = _time_builds(knng, xd, op, flags, args.steps, args.warmup, flush, stream, ws)
    step_s = _max_over_ranks(step_s, ws, device)
    clocks = clk.summary()

    # per-kernel CUDA-event times, recorded by the library on its launching
    # stream, in one more build (events inside a captured graph cannot be
    # timed: this build runs without one)
    flush.fill_(1)
    torch.cuda.synchronize()
    _, _, tst = knng.knng_build(xd, op.K, op.rho, op.delta, op.max_iters, seed=0,
                                flags=(flags & ~knng.FLAG_GRAPH) | knng.FLAG_TIMING)
    torch.cuda.synchronize()

    # end to end through the public API: pinned host input, host outputs
    xh = torch.from_numpy(x).pin_memory()
    oi = torch.empty((w.n, w.K), dtype=torch.int32).pin_memory()
    od = torch.empty((w.n, w.K), dtype=torch.float32).pin_memory()
    e2e = []
    for i in range(args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        _barrier(ws)
        t0 = time.perf_counter()
        knng.knng_build(xh, op.K, op.rho, op.delta, op.max_iters, seed=0, flags=flags, out=(oi, od))
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e.append(t1 - t0)
    e2e_s = _max_over_ranks(sum(e2e) / len(e2e), ws, device)

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    # recall on sampled rows (10,000 from a million points up) against the
    # GPU brute force, for NN-Descent seeds 0 (the timed builds), 1 and 2
    nrows = 10_000 if w.n >= 1_000_000 else RECALL_ROWS
    rows = np.random.default_rng(0).choice(w.n, nrows, replace=False)
    bi, _ = knng.knng_bruteforce(xd, w.K, rows=torch.from_numpy(rows).to(device))
    bi = bi.cpu().numpy()
    rec = metrics.recall(x, ids.cpu().numpy(), bi, rows)
    rec_seeds = [rec]
    for sd in (1, 2):
        si, _, _ = knng.knng_build(xd, op.K, op.rho, op.delta, op.max_iters, seed=sd, flags=flags)
        rec_seeds.append(metrics.recall(x, si.cpu().numpy(), bi, rows))

    def point(p, fl, steps=2):
        t, (pi, _, pst) = _time_builds(knng, xd, p, fl, steps, 1, flush, stream)
        return {"rho": p.rho, "delta": p.delta, "max_iters": p.max_iters, "s": pst["s"],
                "value": round(t, 6), "unit": "s", "recall_at_k": round(metrics.recall(x, pi.cpu().numpy(), bi, rows), 5),
                "iterations": pst["iterations"], "candidates_over_cap": pst["set_overflow"]}

    # the measured ladder (float32 unless --bf16) and the bf16 form beside the
    # float32 one, each with the same rows, flush and protocol (2 timed builds)
    ladder, bf16_form, stated = None, None, None
    if not overridden:
        ladder = [point(dataclasses.replace(op, rho=r, delta=dl, max_iters=it), flags)
                  for (r, dl, it) in LADDER.get(args.workload, [])]
        stated = next((q for q in ladder if (q["rho"], q["delta"], q["max_iters"]) == (w.rho, w.delta, w.max_iters)),
                      None)
        if w.d >= 64 and not (args.bf16 or args.fp8):
            bf16_form = {"at_timed_point": point(op, flags | knng.FLAG_BF16),
                         "at_stated_parameters": point(w, flags | knng.FLAG_BF16),
                         "fp8_at_timed_point": point(op, flags | knng.FLAG_FP8)}

    # the metric's recall condition
    recall_ok = min(rec_seeds) >= 0.99
    reach = {"reached": recall_ok}
    if not recall_ok:
        best = max(ladder or [], key=lambda q: q["recall_at_k"], default=None)
        reach = {"reached": False, "note": "no point of the ladder reaches recall 0.99 on every seed",
                 "best_ladder_point": best}

    peaks = _peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    ran = max(1, tst["join_ran"])
    jname = JOIN_KERNELS.get(tst["join_path"], "join")
    kern = {jname: (join_bytes(tst, dp), tst["join_ms_ran"]),
            "merge_kernel": (merge_bytes(tst), tst["merge_ms_ran"])}
    name = max(kern, key=lambda k: kern[k][1])
    jb = kern[name][0] / ran
    jt = kern[name][1] / 1e3 / ran
    achieved = jb / jt / 1e9
    traffic = measured_traffic(f"{name}@{wname}" + ("+fp8" if args.fp8 else "+bf16" if args.bf16 else ""))
    roof = {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
            "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": traffic,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback",
            "bytes_per_launch": round(jb), "launch_ms": round(jt * 1e3, 4), "launches": ran,
            "launch": "one iteration's local join: the set kernel and every node-range pass of the join "
                      "kernel (list merges excluded), CUDA events on the library's stream",
            "time_share_join_merge_ms": [round(tst["join_ms_ran"], 3), round(tst["merge_ms_ran"], 3)],
            "step_share": round((kern[name][1] / 1e3) / step_s, 3)}
    l2_gbs = knng.measure_l2_read(32 << 20, 200)

    cpu = None
    if not args.no_cpu and ws == 1:
        cpu = cpu_baseline(op, x, wname, step_evals=stats["dist_evals"])

    line = {
        "metric": METRIC, "value": round(step_s, 6), "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 4), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "fp8+f32" if args.fp8 else ("bf16+f32" if args.bf16 else "f32"), "data": "synthetic",
        "config": {"workload": wname, "n": w.n, "d": w.d, "K": w.K, "rho": op.rho, "delta": op.delta,
                   "max_iters": op.max_iters,
                   "stated_parameters": {"rho": w.rho, "delta": w.delta, "max_iters": w.max_iters},
                   "reorder": "parallel" if args.reorder_parallel else ("algorithm1" if args.reorder else False),
                   "bf16": bool(args.bf16), "fp8": bool(args.fp8), "graph": bool(args.graph),
                   "autotune": bool(args.autotune),
                   "join_path": stats["join_path"], "sampler": "heap" if args.heap else "turbo",
                   "parallelism": f"replicas{ws}",
                   "l2": "flushed between timed steps (256 MiB write)", "inputs": "device-resident"},
        "recall_at_k": round(rec, 5), "recall_rows": nrows,
        "recall_seeds_0_1_2": [round(r, 5) for r in rec_seeds],
        "recall_mean_3_seeds": round(sum(rec_seeds) / 3, 5),
        "recall_0.99": reach,
        "stated_parameters": stated,
        "ladder": ladder,
        "bf16_form": bf16_form,
        "iterations": stats["iterations"], "dist_evals": stats["dist_evals"],
        "candidates_over_cap": stats["set_overflow"],
        "selection_ms_per_iter": round(tst["sample_ms_ran"] / ran, 4),
        # the proposal pipeline of the timed point: keys the joins handed to
        # the list merges, and the list insertions they made
        "proposals": {"keys": tst["proposals"], "insertions": tst["inserts"],
                      "keys_per_insertion": round(tst["proposals"] / max(1, tst["inserts"]), 2),
                      "merge_ms_per_iter": round(tst["merge_ms_ran"] / ran, 4)},
        "dist_evals_per_s": round(stats["dist_evals"] / step_s, 1),
        "paper_flops_per_s": round(stats["dist_evals"] * (3 * w.d - 1) / step_s, 1),
        "e2e": {"value": round(e2e_s, 6), "unit": "s", "h2d_bytes_per_step": int(x.nbytes),
                "d2h_bytes_per_step": int(w.n * w.K * 8)},
        "gpu_launches": int(stats["kernel_launches"]) * args.steps,
        "roofline": roof,
        "roofline_l2": {"kernel": name, "bound": "l2", "achieved": round(achieved, 1),
                        "peak": round(l2_gbs, 1), "unit": "GB/s", "frac": round(achieved / l2_gbs, 4),
                        "peak_source": "knng_measure_l2_read: 32 MiB read 200 times in one launch"},
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _oracle_total_evals(wname, op, step_evals):
    """Distance evaluations of one whole build at the timed point: the
    oracle's own count from tests/golden/oracle_recall.json (written by the
    oracle alone) when it holds this point, else the timed build's count."""
    try:
        rec = json.load(open(GOLDEN))[wname]
        if (rec["rho"], rec["delta"], rec["max_iters"], rec["n"]) == (op.rho, op.delta, op.max_iters, op.n):
            return rec["dist_evals"], "the oracle's own count (tests/golden/oracle_recall.json)"
    except Exception:
        pass
    return step_evals, "the timed GPU build's count"


def cpu_baseline(op, x, wname, step_evals, target_s: float = 4.0):
    """The oracle as it stands, timed on this host on bounded samples of the
    workload and scaled to one whole build by distance evaluations:
    - all cores: random init and iteration 1 of the whole point set by the
      batched build on every host thread (t1 s, e1 evaluations), value =
      t1 * E / e1 with E the evaluations of a whole build;
    - one core: the calculation step of iteration 1 for the first nodes
      (about target_s seconds of it), value = t * E / e."""
    import oracle
    E, src = _oracle_total_evals(wname, op, step_evals)
    if op.n <= 200_000:
        # small enough for a whole build on every core
        t0 = time.perf_counter()
        _, _, st = oracle.build_knng_mt(x, op.K, op.rho, op.delta, op.max_iters, seed=0)
        t_all = time.perf_counter() - t0
        allc = {"value": round(t_all, 3), "unit": "s", "cores": st["threads"], "kind": "oracle",
                "sample": f"whole build of the workload on {st['threads']} threads (batched mode)"}
    else:
        t0 = time.perf_counter()
        _, _, st = oracle.build_knng_mt(x, op.K, op.rho, 0.0, 1, seed=0)
        t1 = time.perf_counter() - t0
        allc = {"value": round(t1 * E / st["evals"], 3), "unit": "s", "cores": st["threads"], "kind": "oracle",
                "sample": f"random init and iteration 1 of all {op.n} points on {st['threads']} threads "
                          f"({t1:.2f} s, {st['evals']} distance evaluations), scaled to the {E} evaluations of a "
                          f"whole build ({src})"}
    # one core: part of iteration 1's calculation step
    s = oracle.State(x, op.K, op.rho, seed=0)
    s.init_random()
    s.sample(1)
    u0, ev, t = 0, 0, 0.0
    chunk = max(16, op.n // 2000)
    while t < target_s and u0 < op.n:
        t0 = time.perf_counter()
        r = s.join_range(u0, u0 + chunk)
        t += time.perf_counter() - t0
        ev += r["evals"]
        u0 += chunk
    s.close()
    one = {"value": round(t * E / max(1, ev), 3), "unit": "s", "cores": 1, "kind": "oracle",
           "sample": f"calculation step of iteration 1 for nodes 0..{u0 - 1} on one thread ({t:.2f} s, {ev} "
                     f"distance evaluations), scaled to the {E} evaluations of a whole build ({src})"}
    allc["single_core"] = one
    return allc


def _workload(args):
    """The named workload with the command-line overrides applied (smaller n
    for profiling captures; rho, delta, iteration cap for recall sweeps)."""
    import dataclasses
    w = workloads.WORKLOADS[args.workload]
    over = {k: v for k, v in (("n", args.n), ("rho", args.rho), ("delta", args.delta),
                              ("max_iters", args.max_iters)) if v is not None}
    if over:
        w = dataclasses.replace(w, **over)
    return w, w.data(), (args.workload + "".join(f"_{k}{v}" for k, v in over.items()))


def run_reference(args):
    """The reference arm: the CPU oracle on the same workload and timed point,
    one thread.  Set-up (untimed, once): the oracle's random init and the
    selection step of iteration 1 on the whole point set.  Where a whole
    build takes about two seconds or less (judged from the first block of
    nodes), each step times one whole build.  Otherwise each step times the
    calculation step of the next block of nodes (about two seconds of it) and
    scales it to one whole build by distance evaluations, so the
    --steps/--warmup run stays within a few minutes."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    w, x, wname, op, _ = _op_point(args)
    import oracle
    oracle._load()
    E, src = _oracle_total_evals(wname, op, None)
    s = oracle.State(x, op.K, op.rho, seed=0)
    s.init_random()
    s.sample(1)
    if E is None:
        # no stored count for this point: iteration 1 of the oracle's own
        # build at full size stands for every iteration
        E = sum(len(a) * (len(a) - 1) // 2 + len(a) * len(b) for a, b in zip(*s.samples())) * op.max_iters
        src = "iteration 1's evaluations times the iteration cap (no stored count for this point)"
    chunk = max(16, op.n // 5000)
    t0 = time.perf_counter()
    r = s.join_range(0, chunk)
    probe_s = (time.perf_counter() - t0) * E / max(1, r["evals"])
    if probe_s <= 2.0:
        s.close()
        vals = []
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            oracle.build_knng(x, op.K, op.rho, op.delta, op.max_iters, seed=0)
            if i >= args.warmup:
                vals.append(time.perf_counter() - t0)
        _print_reference(ws, args, w, wname, op, sum(vals) / len(vals),
                         "per step, one whole build of the workload on one thread")
        return
    # the probe block was the first of the sequence: carry on after it
    u0, vals = chunk, []
    for i in range(args.warmup + args.steps):
        t, ev = 0.0, 0
        while t < 2.0:
            if u0 >= op.n:
                s.close()
                s = oracle.State(x, op.K, op.rho, seed=0)
                s.init_random()
                s.sample(1)
                u0 = 0
            t0 = time.perf_counter()
            r = s.join_range(u0, u0 + chunk)
            t += time.perf_counter() - t0
            ev += r["evals"]
            u0 += chunk
        if i >= args.warmup:
            vals.append(t * E / max(1, ev))
    s.close()
    _print_reference(ws, args, w, wname, op, sum(vals) / len(vals),
                     f"per step, the calculation step of iteration 1 for about 2 s of nodes on one thread, scaled "
                     f"to the {E} distance evaluations of a whole build ({src})")


def _print_reference(ws, args, w, wname, op, v, sample):
    """The reference arm's JSON line: the oracle's seconds per build v."""
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v * 1e3, 1),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wname, "n": w.n, "d": w.d, "K": w.K, "rho": op.rho, "delta": op.delta,
                   "max_iters": op.max_iters, "parallelism": "cpu1"},
        "cpu_baseline": {"value": round(v, 3), "unit": "s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--reorder", action="store_true", help="Algorithm 1 relabelling after iteration 1")
    ap.add_argument("--bf16", action="store_true", help="bf16 tensor-core dots for d >= 64, float32 re-rank")
    ap.add_argument("--fp8", action="store_true", help="e4m3 tensor-core dots for d >= 64 (lossy), float32 re-rank")
    ap.add_argument("--graph", action="store_true", help="launch the iteration loop as one captured CUDA graph")
    ap.add_argument("--autotune", action="store_true", help="time the join kernels on the first build, keep the fastest")
    ap.add_argument("--reorder-parallel", action="store_true",
                    help="the parallel relabelling variant after iteration 1")
    ap.add_argument("--heap", action="store_true",
                    help="priority-heap candidate selection instead of Section 3.1's turbosampling")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(workloads.WORKLOADS) + ["batched_256"],
                    help="another workload than the headline one (measurement table)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle timing")
    ap.add_argument("--batched-plain", action="store_true",
                    help="batched workload without the captured graph and the autotuner")
    ap.add_argument("--sweep-d", action="store_true", help="dimension sweep at n=16,384 (one JSON line per run)")
    ap.add_argument("--bruteforce", action="store_true", help="time the exact brute-force K-NNG on the workload")
    ap.add_argument("--rows", type=int, default=0, help="brute force: sampled query rows (0 = every row)")
    ap.add_argument("--relabel-ab", action="store_true",
                    help="no relabelling vs Algorithm 1 vs the parallel variant (one JSON line each)")
    ap.add_argument("--n", type=int, default=None, help="override the workload's point count (profiling)")
    ap.add_argument("--rho", type=float, default=None, help="override the sample rate (recall sweeps)")
    ap.add_argument("--delta", type=float, default=None, help="override the termination threshold")
    ap.add_argument("--max-iters", type=int, default=None, help="override the iteration cap")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        print("note: at least 3 warm-up steps are required; using 3", file=sys.stderr)
        args.warmup = 3
    if args.sweep_d:
        run_sweep(args)
    elif args.bruteforce and args.impl == "gb300":
        run_bruteforce(args)
    elif args.relabel_ab and args.impl == "gb300":
        run_relabel_ab(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched_256":
        if any(v is not None for v in (args.n, args.rho, args.delta, args.max_iters)):
            ap.error("--n/--rho/--delta/--max-iters do not apply to the batched workload")
        run_batched(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
