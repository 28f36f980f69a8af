#!/usr/bin/env python
"""Throughput of S_k(A) evaluation on GB300, one JSON line on stdout.

Default workload (the precision form): n = 8192, planted symmetric spectrum
lam ~ U[-0.97, 0.97], k = 3375 = 15^3 by the radix-15 kernel in the residual
framework, products on the tcgen05 tensor cores from split hi+lo BF16
operands. A step is one evaluation (16 products and their fused epilogues).
The line also reports repeated squaring (k = 4096, the paper's binary
comparator) on the same input and arithmetic.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Under torchrun every rank evaluates its own replica (independent seeds); the
evaluations do not communicate ("replicas only"), so scaling is weak.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "S_k(A) evals/s & % tensor peak: radix-15/9 vs squaring, split-BF16 vs FP64"
UNIT = "S_k/s"

# steps: the default number of timed steps, sized so that the timed region lasts about 2 s on
# one GB300 (the products' power-capped regime, where the sustained peak is measured).
WORKLOADS = {
    "precision-r15-bf16-n8192-k3375": dict(steps=64, cfg=3, n=8192, k=3375, radix=15, dtype="split_bf16", sq_k=4096),
    "precision-r9-bf16-n8192-k6561": dict(steps=56, cfg=3, n=8192, k=6561, radix=9, dtype="split_bf16", sq_k=8192),
    "precision-r15-fp16-n8192-k3375": dict(steps=64, cfg=3, n=8192, k=3375, radix=15, dtype="split_fp16", sq_k=4096),
    "precise-r15-fp16-n8192-k3375": dict(steps=44, cfg=3, n=8192, k=3375, radix=15, dtype="split_fp16", sq_k=4096,
                                         precise=True),
    "precise-r15-bf16-n8192-k3375": dict(steps=44, cfg=3, n=8192, k=3375, radix=15, dtype="split_bf16", sq_k=4096,
                                         precise=True),
    # the same symmetric input through NEUMANN_FLAG_SYMMETRIC: products compute the tiles on or
    # above the diagonal only, so the roofline counts that work, not 2 n^3
    "symmetric-r15-bf16-n8192-k3375": dict(steps=108, cfg=3, n=8192, k=3375, radix=15, dtype="split_bf16", sq_k=4096,
                                           symmetric=True),
    "symmetric-r15-fp16-n8192-k3375": dict(steps=108, cfg=3, n=8192, k=3375, radix=15, dtype="split_fp16", sq_k=4096,
                                           symmetric=True),
    "precision-r9-fp16-n8192-k6561": dict(steps=56, cfg=3, n=8192, k=6561, radix=9, dtype="split_fp16", sq_k=8192),
    # five-product kernels (radix 24, 25: 7 products per level) on the same input
    "precision-r25-bf16-n8192-k15625": dict(steps=48, cfg=3, n=8192, k=15625, radix=25, dtype="split_bf16", sq_k=16384),
    "precision-r24-bf16-n8192-k13824": dict(steps=48, cfg=3, n=8192, k=13824, radix=24, dtype="split_bf16", sq_k=16384),
    # approximate-prefix five-product kernels (App. C, Table approx): k = 27^3, 31^3
    "precision-r27-bf16-n8192-k19683": dict(steps=48, cfg=3, n=8192, k=19683, radix=27, dtype="split_bf16", sq_k=16384),
    "precision-r31-bf16-n8192-k29791": dict(steps=48, cfg=3, n=8192, k=29791, radix=31, dtype="split_bf16", sq_k=32768),
    # cfg 5: n = 16384, planted spectrum U[-0.95, 0.95] + rank-32 nonsymmetric term of norm 0.01;
    # the FP64 comparison (about two minutes at this size) runs only with --fp64-large
    "large-r15-fp16-n16384-k3375": dict(steps=8, cfg=5, n=16384, k=3375, radix=15, dtype="split_fp16", sq_k=4096,
                                        fp64=False),
    "large-precise-r15-fp16-n16384-k3375": dict(steps=6, cfg=5, n=16384, k=3375, radix=15, dtype="split_fp16",
                                                sq_k=4096, fp64=False, precise=True),
    "plain-r9-fp32-n4096-k729": dict(steps=50, cfg=2, n=4096, k=729, radix=9, dtype="fp32", sq_k=1024),
    "plain-r15-fp32-n4096-k225": dict(steps=64, cfg=2, n=4096, k=225, radix=15, dtype="fp32", sq_k=256),
    # the default workload's input and k through the plain FP32 path (SIMT products)
    "plain-r15-fp32-n8192-k3375": dict(steps=3, cfg=3, n=8192, k=3375, radix=15, dtype="fp32", sq_k=4096),
    "plain-r9-fp64-n4096-k729": dict(steps=3, cfg=2, n=4096, k=729, radix=9, dtype="fp64", sq_k=1024),
    # cfg 4: 4096 damped-Jacobi matrices, n uniform in {16, 32, ..., 256}; a step is one
    # grouped evaluation of the whole batch
    "batched-r9-bf16-4096-k81": dict(steps=160, cfg=4, count=4096, k=81, radix=9, dtype="split_bf16", batched=True),
    "batched-r15-bf16-4096-k225": dict(steps=130, cfg=4, count=4096, k=225, radix=15, dtype="split_bf16", batched=True),
    "batched-r9-fp32-4096-k81": dict(steps=90, cfg=4, count=4096, k=81, radix=9, dtype="fp32", batched=True),
    "batched-r15-fp32-4096-k225": dict(steps=64, cfg=4, count=4096, k=225, radix=15, dtype="fp32", batched=True),
    "batched-r25-bf16-4096-k625": dict(steps=76, cfg=4, count=4096, k=625, radix=25, dtype="split_bf16", batched=True),
    # the same construction restricted to orders 16..64: the batch the resident launch serves
    "batched-small-r9-bf16-4096-k81": dict(steps=200, cfg=4, count=4096, k=81, radix=9, dtype="split_bf16",
                                           batched=True, sizes=(16, 32, 48, 64)),
}
DEFAULT_WORKLOAD = "precision-r15-bf16-n8192-k3375"

# DRAM bytes (read + write) per launch of the tensor-core product, the mean over
# the 16 launches of one evaluation of the named workload, from one ncu capture
# (profiles/tc_split_gemm_n8192_r15_bench.md). Valid for the kernel and schedule
# sources whose SHA-1 prefix (of the code without comments) is recorded beside
# it; reported as null otherwise.
TC_TRAFFIC = {"sha1": "9f28e5d9487a", "workload": "precision-r15-bf16-n8192-k3375", "bytes_per_launch": 3.9885e9}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


_PEAKS_LIVE = {}


def live_peaks(dev):
    """Denominators that MEASURED_PEAKS.json does not hold, measured on this
    device in this run (no clock or setting is changed):
      sms               the device's SM count
      fp32_tflops       CUDA-core FP32 FMA rate (neumann_measure_fma_peak: timed
      fp64_tflops       launches of independent FMA chains on every SM), FP64 likewise
      fp16_over_bf16    cuBLAS FP16 / BF16 dense GEMM rate at 8192^3 (torch.matmul,
                        best of 5 each, CUDA events), the factor that turns the
                        measured BF16 tensor peak into the FP16 one
    """
    if dev in _PEAKS_LIVE:
        return _PEAKS_LIVE[dev]
    import torch

    import paper_2602_11843_gb300 as nm

    stream = torch.cuda.current_stream(dev)
    f32, sms = nm.neumann_measure_fma_peak(nm.FP32, stream.cuda_stream)
    f64, _ = nm.neumann_measure_fma_peak(nm.FP64, stream.cuda_stream)
    rates = {}
    n = 8192
    for name, dt in (("bf16", torch.bfloat16), ("fp16", torch.float16)):
        a = torch.randn((n, n), device=dev, dtype=dt)
        b = torch.randn((n, n), device=dev, dtype=dt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = None
        for rep in range(6):
            e0.record(stream)
            torch.matmul(a, b)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if rep:
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
        rates[name] = 2.0 * n ** 3 / (best / 1e3) / 1e12
        del a, b
    out = {"sms": sms, "fp32_tflops": f32, "fp64_tflops": f64,
           "bf16_tflops_torch_burst": rates["bf16"], "fp16_tflops_torch_burst": rates["fp16"],
           "fp16_over_bf16": rates["fp16"] / rates["bf16"]}
    _PEAKS_LIVE[dev] = out
    return out


def _code_only(text):
    """C++/CUDA source without its comments and blank lines: edits to comments
    leave the key of a captured kernel unchanged."""
    import re

    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*$", "", line).rstrip() for line in text.splitlines())
    return "\n".join(line for line in lines if line)


def _src_sha(*names):
    h = hashlib.sha1()
    for name in names:
        with open(os.path.join(ROOT, "paper_2602_11843_gb300", "csrc", name)) as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:12]


def reduce_max_ms(ms, world, device=None):
    """The job time: the maximum over ranks of each rank's timed region (ms)."""
    if world == 1:
        return float(ms)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank_step, steps, world, ms_max):
    """Whole-job throughput: the units every rank processed over the job time."""
    return units_per_rank_step * steps * world / (ms_max / 1e3)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples (200 ms) of this GPU's clocks and throttle reasons.

    The sampler starts before the timed region and stops after it; summary() keeps
    the samples whose nvidia-smi timestamp falls inside the region (from entering
    the `with` block to leaving it)."""

    FIELDS = ("timestamp,index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.t0 = self.t1 = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        self.t0 = time.time()
        return self

    def __exit__(self, *exc):
        self.t1 = time.time()
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    @staticmethod
    def _stamp(text):
        import datetime

        try:
            return datetime.datetime.strptime(text, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def summary(self):
        self.tmp.flush()
        rows = []
        try:
            with open(self.tmp.name) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) < 11:
                        continue
                    if self.uuid and self.uuid not in parts[2]:
                        continue
                    rows.append(parts)
        finally:
            os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        inside = [r for r in rows if (t := self._stamp(r[0])) is not None and self.t0 <= t <= self.t1]
        note = None
        if not inside:  # a region shorter than the sampling interval
            inside, note = rows, "no sample inside the timed region: all samples of the run"

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[3]) for r in inside if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[7 + i].lower().startswith("active")})
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(inside[0][4]),
               "power_w_max": max((num(r[5]) or 0.0) for r in inside), "samples": len(inside),
               "region_s": round(self.t1 - self.t0, 3), "reasons": reasons}
        if note:
            out["note"] = note
        return out


_INPUTS = {}


def make_input(wl, seed_rep):
    from workloads import generators as G

    key = (wl["cfg"], seed_rep, wl["n"])
    if key not in _INPUTS:
        _INPUTS.clear()  # one workload's input at a time (n = 16384 holds 2 GB)
        _INPUTS[key] = G.config_inputs(wl["cfg"], r=seed_rep, n=wl["n"])
    return _INPUTS[key]


def cpu_baseline(wl, A_np, budget_products=None):
    """The oracle as it stands, on a bounded sample: the first `p` products of the
    same scheme at the same n (FP64, NumPy/BLAS on the host cores), scaled to
    S_k/s by the oracle's product count for the whole evaluation."""
    import numpy as np

    from oracle import circuits as C
    from oracle import evaluate as EV
    from oracle import schemes as SC

    n = A_np.shape[0]
    alg = C.matrix_algebra(n)
    ks = EV.kernels()
    levels = SC.pure_levels(wl["k"], wl["radix"])
    count_alg = C.matrix_algebra(2)
    (SC.radix_residual if wl["radix"] in EV.APPROX else SC.radix_exact)(np.eye(2), levels, ks, count_alg)
    total = count_alg.products
    t0 = time.perf_counter()
    ks[wl["radix"]](A_np, alg)  # first level's kernel: mu_m products of the oracle
    dt = time.perf_counter() - t0
    per_product = dt / alg.products
    return {"value": 1.0 / (per_product * total), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "extrapolated": f"{alg.products} of {total} products timed, scaled to {total}",
            "sample": f"first-level radix-{wl['radix']} kernel ({alg.products} of {total} products) at n={n}, "
                      f"FP64 NumPy/BLAS, scaled by product count; {dt:.1f} s"}


def oracle_error(wl, inp, S_np):
    """CPU-baseline leg, second part: the oracle's FP64 result for the same input
    (closed form on the planted spectrum: S_k for exact radices, Lemma 5.7's value
    for radix 15, 24, 25) and the GPU result's relative Frobenius error against it."""
    from oracle import closed_form as CF
    from oracle import evaluate as EV

    if "V" not in inp or "X" in inp:  # no closed form (the perturbed n = 16384 input)
        return None
    t0 = time.perf_counter()
    ref = EV.planted_reference(inp["V"], inp["lam"], wl["k"], wl["radix"])
    err = CF.rel_fro(S_np, ref)
    out = {"rel_fro": err, "reference": "oracle closed form, FP64 (" +
           ("Lemma 5.7 framework value" if wl["radix"] in EV.APPROX else "S_k") + ")",
           "host_s": round(time.perf_counter() - t0, 1)}
    if wl["radix"] in EV.APPROX:
        out["framework_vs_sk"] = CF.rel_fro(ref, EV.planted_reference(inp["V"], inp["lam"], wl["k"], 1))
    return out


def oracle_error_batched(wl, mats, outs, every=64):
    """CPU-baseline leg for a batch: every `every`-th matrix against the oracle's
    matrix scheme (FP64); the largest and median relative Frobenius error."""
    import numpy as np

    from oracle import closed_form as CF
    from oracle import evaluate as EV

    errs = [CF.rel_fro(outs[i].double().cpu().numpy(), EV.evaluate(mats[i]["A"], wl["k"], wl["radix"])[0])
            for i in range(0, len(mats), every)]
    return {"max_rel_fro": float(np.max(errs)), "median_rel_fro": float(np.median(errs)),
            "matrices_checked": len(errs), "reference": "oracle matrix scheme, FP64"}


def run_reference(args, wl):
    """--impl reference: the CPU oracle timed on the host cores (rank 0 only)."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    import numpy as np

    from oracle import circuits as C
    from oracle import evaluate as EV

    if wl.get("batched"):
        from workloads import generators as G

        mats = G.jacobi_batch(wl["count"], 1000 * wl["cfg"])
        times = []
        for it in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            done = 0
            for m in mats[it * 8 % len(mats):]:
                EV.evaluate(m["A"], wl["k"], wl["radix"])
                done += 1
                if done >= 8:
                    break
            if it >= args.warmup:
                times.append((time.perf_counter() - t0) / done)
        value = 1.0 / statistics.median(times)
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * len(mats) / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "count": len(mats), "k": wl["k"], "radix": wl["radix"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "each step: 8 matrices of the batch, scaled to S_k/s"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    inp = make_input(wl, 0)
    A = np.asarray(inp["A"], dtype=np.float64)
    ks = EV.kernels()
    info_products = None
    times = []
    for it in range(args.warmup + args.steps):
        alg = C.matrix_algebra(A.shape[0])
        t0 = time.perf_counter()
        ks[wl["radix"]](A, alg)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt / alg.products)
        info_products = alg.products
    from oracle import schemes as SC

    calg = C.matrix_algebra(2)
    levels = SC.pure_levels(wl["k"], wl["radix"])
    (SC.radix_residual if wl["radix"] in EV.APPROX else SC.radix_exact)(np.eye(2), levels, ks, calg)
    per_eval = statistics.median(times) * calg.products
    value = 1.0 / per_eval
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_eval * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": wl["n"], "k": wl["k"], "radix": wl["radix"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"each step: one radix-{wl['radix']} kernel ({info_products} products) at "
                                   f"n={wl['n']}, scaled to a full evaluation ({calg.products} products)",
                         "extrapolated": f"{info_products} of {calg.products} products timed, scaled to "
                                         f"{calg.products}"},
        "extrapolated": f"{info_products} of {calg.products} products timed per step, scaled to {calg.products}",
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched(args, wl, sub=False):
    """cfg 4: one grouped evaluation of the whole batch per step; compared with the
    same batch evaluated one matrix (one plan, its own launches) at a time.
    sub: a secondary workload of the default run (one process): returns its line."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2602_11843_gb300 as nm
    from workloads import generators as G

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if sub:
        world = 1
    elif world > 1:
        dist.init_process_group("nccl", device_id=dev)
    mats = G.jacobi_batch(wl["count"], 1000 * wl["cfg"] + rank, **({"sizes": wl["sizes"]} if "sizes" in wl else {}))
    ns = [m["n"] for m in mats]
    bflags = nm.FLAG_TIMING | (nm.FLAG_NO_RESIDENT if args.no_resident else 0)
    bp = nm.BatchedPlan(len(mats), 256, wl["k"], wl["radix"], wl["dtype"], bflags)
    dt = torch.float32 if wl["dtype"] == "fp32" else torch.float64
    # the batch lives in one contiguous buffer (A_i are views), so an end-to-end
    # step moves it with one copy each way
    offs = np.cumsum([0] + [n * n for n in ns])
    A_all = torch.empty(int(offs[-1]), dtype=dt, device=dev)
    S_all = torch.empty_like(A_all)
    host = np.concatenate([m["A"].reshape(-1) for m in mats])
    A_all.copy_(torch.from_numpy(host).to(dt))
    As = [A_all[offs[i]:offs[i + 1]].view(n, n) for i, n in enumerate(ns)]
    outs = [S_all[offs[i]:offs[i + 1]].view(n, n) for i, n in enumerate(ns)]
    if not args.no_autotune:
        bp.autotune(As, outs, reps=2)  # the library's autotuner picks the matrices per pass
    bp.bind(As, outs)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        bp.launch()
    torch.cuda.synchronize()
    nm.neumann_plan_timing(bp.handle, 1 << 16)
    assert bp.status() == 0
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(uuid) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            bp.launch()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if world > 1:
        dist.barrier()
    ms_max = reduce_max_ms(ms, world, dev)
    prod_ms = nm.neumann_plan_timing(bp.handle, 1 << 16)
    status = bp.status()
    value = job_value(len(mats), args.steps, world, ms_max)
    info = nm.neumann_plan_info(bp.handle)
    ck = info["batch_chunk"] or len(mats)
    nres = sum(1 for x in ns if x <= info["resident_max_n"])
    # launches per step: each op of the scheme once per grouped pass, plus the resident launch
    launches = info["launches"] * ((len(mats) - nres + ck - 1) // ck) + (1 if nres else 0)
    # the same step captured once in a CUDA graph and replayed (resident and grouped launches)
    graph = None
    try:
        gp = nm.BatchedPlan(len(mats), 256, wl["k"], wl["radix"], wl["dtype"],
                            nm.FLAG_NO_RESIDENT if args.no_resident else 0)
        gp.bind(As, outs)  # created after bp's tuning: it starts from the same tuned configuration
        gs = torch.cuda.Stream(dev)
        with torch.cuda.stream(gs):
            gp.launch()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=gs):
            gp.launch()
        g.replay()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        gms = e0.elapsed_time(e1) / args.steps
        graph = {"ms_per_step": gms, "value": job_value(len(mats), args.steps, 1, gms * args.steps), "unit": UNIT}
    except Exception as ex:  # noqa: BLE001 - reported, not fatal
        graph = {"error": str(ex)[:200]}
    # the same batch, one plan per matrix order and one evaluation (own launches) per matrix
    plans = {}
    for n in sorted(set(ns)):
        plans[n] = nm.Plan(n, wl["k"], wl["radix"], wl["dtype"])
    for a, o in zip(As, outs):
        plans[a.shape[0]](a, out=o)
    torch.cuda.synchronize()
    e0.record(stream)
    for a, o in zip(As, outs):
        plans[a.shape[0]](a, out=o)
    e1.record(stream)
    torch.cuda.synchronize()
    per_matrix_ms = e0.elapsed_time(e1)
    # end to end through the C ABI's packed host-batch call (neumann_eval_batched_host):
    # every step copies the pinned packed batch in and the results out; the library
    # overlaps the copies with the neighbouring steps' evaluations. Host wall clock
    # from the first call to the last result in host memory.
    A_host = A_all.cpu().pin_memory()
    S_host = torch.empty_like(A_host).pin_memory()
    h2d = A_host.numel() * A_host.element_size()
    bp.eval_host(ns, A_host, S_host)
    bp.host_wait()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        bp.eval_host(ns, A_host, S_host)
    bp.host_wait()
    e2e_value = job_value(len(mats), args.steps, world, reduce_max_ms((time.perf_counter() - t0) * 1e3, world, dev))
    nm.neumann_plan_timing(bp.handle, 1 << 16)
    peaks, peak_src = _peaks()
    tc = wl["dtype"].startswith("split")
    per = info["products_executed"]
    # the grouped product kernel's work: the matrices the resident launch does not take
    gns = [x for x in ns if x > info["resident_max_n"]]
    flops_one = sum(2.0 * n ** 3 for n in gns)  # one product over the grouped matrices, 2 n^3 each
    mean_prod = statistics.mean(prod_ms) if prod_ms else float("nan")
    # The products of orders <= 256 have little arithmetic per byte (about n / 5
    # tensor flops per byte), so both rooflines are computed and the one that
    # bounds the product (the longer ideal time) is reported.
    prod_s = sum(prod_ms) / args.steps / 1e3  # product time per step
    bytes_step = sum(n * n for n in gns) * info["product_bytes_per_element"]
    flops_step = per * flops_one * (3 if tc else 1)
    live = live_peaks(dev)
    fpeak = peaks["bf16_tflops_sustained"] if tc else live["fp32_tflops"]
    hbm = {"bound": "hbm", "achieved": bytes_step / prod_s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "peak_source": f"hbm_gbs ({peak_src})",
           "work_per_launch": "algorithmic bytes: sum n_i^2 x the product's input, output and operand bytes per "
                              f"element ({info['product_bytes_per_element']} B over the {per} products)"}
    alu = {"bound": "tensor" if tc else "alu", "achieved": flops_step / prod_s / 1e12, "peak": fpeak,
           "unit": "TFLOP/s",
           "peak_source": f"bf16_tflops_sustained ({peak_src})" if tc else
                          "FP32 FMA rate measured in this run (neumann_measure_fma_peak)",
           "work_per_launch": "3 x sum 2 n_i^3 BF16 tensor flops" if tc else "sum 2 n_i^3 FP32 flops"}
    t_hbm = bytes_step / (hbm["peak"] * 1e9)
    t_alu = flops_step / (alu["peak"] * 1e12)
    roof = dict(hbm if t_hbm >= t_alu else alu)
    other = alu if t_hbm >= t_alu else hbm
    roof["other"] = {"bound": other["bound"], "achieved": other["achieved"], "peak": other["peak"],
                     "unit": other["unit"], "frac": other["achieved"] / other["peak"]}
    roof["traffic"] = None
    roof["kernel"] = "tc_split_gemm_kernel (grouped)" if tc else "simt_gemm_kernel (grouped)"
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["effective_tflops"] = per * flops_one / prod_s / 1e12
    roof["launches_timed"] = len(prod_ms)
    if prod_ms and per and len(prod_ms) % per == 0:
        reps = len(prod_ms) // per
        roof["per_product_ms"] = [round(sum(prod_ms[i::per]) / reps, 4) for i in range(per)]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if tc else "f32",
        "precision": "hi+lo BF16 operands, 3 products, FP32 accumulate, FP64 Y and R" if tc else
                     "FP32 products, FP64 Y and R",
        "data": "synthetic",
        "config": {"workload": args.workload, "count": len(mats),
                   "n": "uniform in {%s}" % ",".join(map(str, wl.get("sizes", range(16, 257, 16)))), "k": wl["k"],
                   "radix": wl["radix"], "scheme": wl["dtype"], "products_per_matrix": per,
                   "launches_per_step": launches,
                   "batch_chunk": info["batch_chunk"], "autotuned": bool(info["tuned"]),
                   "resident_max_n": info["resident_max_n"],
                   "resident_matrices": nres,
                   "l2": "inputs larger than L2 (the batch's A alone is 0.39 GB in FP32)",
                   "parallelism": f"replicas x{world}"},
        "vs_per_matrix": {"ms_per_batch": per_matrix_ms, "speedup": per_matrix_ms / (ms_max / args.steps)},
        "graph_replay": graph,
        "status": status, "clocks": clk.summary(),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d},
        "gpu_launches": args.steps * launches,
        "roofline": roof,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if not sub:
            line["cpu_baseline"] = cpu_baseline_batched(wl, mats)
        bp.launch()  # the outputs last held the per-matrix comparison's results
        torch.cuda.synchronize()
        line["vs_oracle"] = oracle_error_batched(wl, mats, outs)
    if sub:
        return line
    line["peaks_measured_here"] = live_peaks(dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    del np


def cpu_baseline_batched(wl, mats, budget_s=10.0):
    """The oracle on the host cores: the same scheme on matrices of the batch, one
    after another, for about `budget_s` seconds, scaled to S_k/s."""
    from oracle import evaluate as EV

    t0 = time.perf_counter()
    done = 0
    for m in mats:
        EV.evaluate(m["A"], wl["k"], wl["radix"])
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"first {done} of {len(mats)} matrices (same order of draw), FP64 NumPy; {dt:.1f} s"}


def run_ours(args, wl, sub=False):
    """One single-matrix workload. sub: a secondary workload of the default run
    (one process, no FP64 comparison, no CPU timing): returns its line."""
    if wl.get("batched"):
        return run_batched(args, wl, sub)
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2602_11843_gb300 as nm

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if sub:
        world = 1
    elif world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    inp = make_input(wl, rank)
    A_np = np.asarray(inp["A"], dtype=np.float64)
    n, k = wl["n"], wl["k"]
    pflags = (nm.FLAG_PRECISE_ACC if wl.get("precise") else 0) | (nm.FLAG_SYMMETRIC if wl.get("symmetric") else 0)
    plan = nm.Plan(n, k, wl["radix"], wl["dtype"], nm.FLAG_TIMING | pflags)
    io = plan.io_dtype
    A = torch.tensor(A_np, dtype=io, device=dev)
    S = torch.empty_like(A)
    stream = torch.cuda.current_stream(dev)
    if args.launch:
        plan.set_launch(*args.launch)  # a hand-set launch configuration instead of the autotuner's
    elif not args.no_autotune:
        plan.autotune(A, out=S, reps=2)  # the library's autotuner picks tiles and raster
    for _ in range(args.warmup):
        plan(A, out=S)
    torch.cuda.synchronize()
    plan.timing()  # discard warm-up and tuning records
    assert plan.status() == 0, "device status set during warm-up"

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(uuid) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            plan(A, out=S)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms_max = reduce_max_ms(ev0.elapsed_time(ev1), world, dev)
    prod_ms = plan.timing()
    status = plan.status()
    info = plan.info
    value = job_value(1, args.steps, world, ms_max)

    # repeated squaring on the same input and arithmetic (the paper's binary comparator)
    sq = nm.Plan(n, wl["sq_k"], 2, wl["dtype"], pflags)
    if args.launch:
        sq.set_launch(*args.launch)
    for _ in range(args.warmup):
        sq(A, out=S)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sq(A, out=S)
    e1.record(stream)
    torch.cuda.synchronize()
    sq_ms = e0.elapsed_time(e1) / args.steps

    # the plain FP64 path on the same input: one evaluation (GB300 runs FP64 at
    # 1/64 of the FP32 rate, so this takes seconds), and the split result's
    # relative Frobenius distance from it
    fp64 = None
    if not sub and wl["dtype"] != "fp64" and not args.no_fp64 and (wl.get("fp64", True) or args.fp64_large):
        p64 = nm.Plan(n, k, wl["radix"], "fp64")
        A64 = A.double() if A.dtype != torch.float64 else A
        S64 = torch.empty_like(A64)
        e0.record(stream)
        p64(A64, out=S64)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_ms = e0.elapsed_time(e1)
        plan(A, out=S)
        torch.cuda.synchronize()
        diff = float(torch.linalg.norm(S.double() - S64) / torch.linalg.norm(S64))
        fp64 = {"ms_per_step": fp64_ms, "speedup": fp64_ms / (ms_max / args.steps), "rel_fro_vs_fp64": diff,
                "products": p64.info["products_executed"]}
        if "probes" in inp:  # cfg 5: the split result on the 64 probe vectors, against the FP64 path's
            X = torch.tensor(inp["probes"], dtype=torch.float64, device=dev)
            SX64 = S64 @ X
            fp64["probe_rel_err_vs_fp64"] = float(torch.linalg.norm(S.double() @ X - SX64) / torch.linalg.norm(SX64))
        del p64, A64, S64

    # cfg 5: the telescoping property on the probes, (I - A) S_k X = X - A^k X with
    # A^k X ~ 0 (rho(A)^k ~ 0.95^3375): relative residual || (I - A)(S X) - X || / || X ||
    probes = None
    if "probes" in inp:
        plan(A, out=S)
        torch.cuda.synchronize()
        X = torch.tensor(inp["probes"], dtype=torch.float64, device=dev)
        SX = S.double() @ X
        resid = SX - A.double() @ SX - X
        probes = {"count": X.shape[1], "telescoping_residual": float(torch.linalg.norm(resid) / torch.linalg.norm(X))}

    # end to end through the C ABI's host-buffer call (neumann_eval_host): every
    # step copies pinned host A in and the result S out; the library overlaps one
    # step's copies with the neighbouring steps' evaluations. Host wall clock
    # from the first call to the last result in host memory.
    A_host = torch.tensor(A_np, dtype=io).pin_memory()
    S_host = torch.empty_like(A_host).pin_memory()
    for _ in range(max(1, args.warmup)):
        plan.eval_host(A_host, out=S_host)
    plan.host_wait()
    torch.cuda.synchronize()
    plan.timing()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.eval_host(A_host, out=S_host)
    plan.host_wait()
    e2e_ms = (time.perf_counter() - t0) * 1e3
    e2e_value = job_value(1, args.steps, world, reduce_max_ms(e2e_ms, world, dev))
    plan.timing()

    peaks, peak_src = _peaks()
    tc = wl["dtype"].startswith("split")
    mean_prod_ms = statistics.mean(prod_ms) if prod_ms else float("nan")
    if tc:
        flops = 3 * 2.0 * n ** 3  # three BF16 products per split product
        work = "3 x 2n^3 BF16 tensor flops"
        if wl.get("symmetric"):  # the 256 x 256 tiles on or above the diagonal only
            t = info["padded_n"] // 256
            flops = 3 * 2.0 * info["padded_n"] * 256 * 256 * (t * (t + 1) // 2)
            work = "3 x 2 x padded_n x 256^2 x (tiles on or above the diagonal) BF16 tensor flops"
        peak = peaks["bf16_tflops_sustained"]
        peak_source = f"bf16_tflops_sustained ({peak_src})"
        if wl["dtype"] == "split_fp16":  # FP16 operands: the BF16 figure x the measured cuBLAS FP16/BF16 ratio
            r = live_peaks(dev)["fp16_over_bf16"]
            peak *= r
            peak_source += f" x {r:.3f} (cuBLAS FP16 / BF16 GEMM rate measured in this run)"
        sha = _src_sha("kernels_tc.cu", "epilogue.cuh", "plan.cpp")  # plan.cpp: the ops' inputs and outputs
        traffic = (TC_TRAFFIC["bytes_per_launch"]
                   if TC_TRAFFIC["sha1"] == sha and args.workload == TC_TRAFFIC["workload"] else None)
        roof = {"bound": "tensor", "achieved": flops / (mean_prod_ms / 1e3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "frac": None, "traffic": traffic,
                "kernel": "tc_split_gemm_kernel", "peak_source": peak_source,
                "work_per_launch": work, "launches_timed": len(prod_ms)}
    else:
        flops = 2.0 * n ** 3
        # CUDA-core FMA rate measured in this run (FP32 or FP64 chains on every SM)
        live = live_peaks(dev)
        peak = live["fp32_tflops"] if wl["dtype"] == "fp32" else live["fp64_tflops"]
        roof = {"bound": "alu", "achieved": flops / (mean_prod_ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": None, "traffic": None, "kernel": "simt_gemm_kernel",
                "peak_source": f"{wl['dtype'].upper()} FMA rate measured in this run (neumann_measure_fma_peak, "
                               f"{live['sms']} SMs)",
                "work_per_launch": "2n^3 flops", "launches_timed": len(prod_ms)}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # mean device time of each product of an evaluation, in launch order
    per = info["products_executed"]
    if prod_ms and per and len(prod_ms) % per == 0:
        reps = len(prod_ms) // per
        roof["per_product_ms"] = [round(sum(prod_ms[i::per]) / reps, 4) for i in range(per)]
    roof["effective_tflops"] = 2.0 * n ** 3 / (mean_prod_ms / 1e3) / 1e12

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"split_bf16": "bf16", "split_fp16": "f16", "fp32": "f32", "fp64": "f64"}[wl["dtype"]],
        "precision": {"split_bf16": "hi+lo BF16 operands, 3 products, FP32 accumulate, FP64 Y and R",
                      "split_fp16": "hi+lo FP16 operands of x*2^e (e per matrix), 3 products, FP32 accumulate, FP64 Y and R",
                      "fp32": "FP32 products, FP64 Y and R", "fp64": "FP64"}[wl["dtype"]]
                     + ("; K accumulated in chunks of 512 summed with round-to-nearest" if pflags else ""),
        "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "k": k, "radix": wl["radix"], "scheme": wl["dtype"],
                   "products_per_step": info["products_executed"], "products_formula": info["products_formula"],
                   "l2": "inputs larger than L2 (A, S and every workspace matrix exceed 129 MB)",
                   "tiles": None if wl["dtype"] in ("fp32", "fp64") else
                            "2-CTA 256x256, upper triangle mirrored" if wl.get("symmetric") else
                            "2-CTA 256x128, chunked accumulation" if pflags else
                            ("2-CTA 256x256" if info["tile_pair"] else "1-CTA 128x256"),
                   "raster_group": info["raster_group"] or None,
                   "autotuned": bool(info["tuned"]) and not args.launch,
                   "parallelism": f"replicas x{world}"},
        "vs_squaring": {"k": wl["sq_k"], "ms_per_step": sq_ms, "speedup": sq_ms / (ms_max / args.steps),
                        "products_executed": sq.info["products_executed"],
                        "formula_ratio": sq.info["products_formula"] / info["products_formula"]},
        "vs_fp64": fp64,
        "probes": probes,
        "status": status,
        "clocks": clk.summary(),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": A_host.numel() * A_host.element_size(),
                "d2h_bytes_per_step": S_host.numel() * S_host.element_size()},
        "gpu_launches": args.steps * info["launches"],
        "roofline": roof,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if not sub:
            line["cpu_baseline"] = cpu_baseline(wl, A_np)
        plan(A, out=S)  # S last held the squaring comparator's result
        torch.cuda.synchronize()
        line["vs_oracle"] = oracle_error(wl, inp, S.double().cpu().numpy())
    if sub:
        return line
    line["peaks_measured_here"] = live_peaks(dev)
    if world == 1 and args.workload == DEFAULT_WORKLOAD and not args.no_extras:
        del plan, sq, A, S, A_host, S_host
        torch.cuda.empty_cache()
        line.update(run_extras(args))
        line["vs_fp32"] = vs_fp32(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# Secondary workloads of the default run, each timed like its own --workload run
# over a shorter region (steps), reported as keys of the default line.
EXTRAS = (("radix9", "precision-r9-bf16-n8192-k6561", 20), ("precise", "precise-r15-bf16-n8192-k3375", 16),
          ("batched", "batched-r9-bf16-4096-k81", 48), ("fp32", "plain-r15-fp32-n8192-k3375", 3))


def vs_fp32(line):
    """The split forms against the plain FP32 path on the same input and k, each
    with its error against the oracle: whether they are faster at an error no
    larger than the FP32 path's."""
    f = line.get("fp32")
    if not f:
        return None

    def err(d):
        return (d.get("vs_oracle") or {}).get("rel_fro")

    pr = line.get("precise", {})
    return {"fp32_value": f["value"], "fp32_rel_fro": err(f),
            "split_value": line["value"], "split_rel_fro": err(line),
            "precise_value": pr.get("value"), "precise_rel_fro": err(pr),
            "speedup_split": line["value"] / f["value"],
            "speedup_precise": pr["value"] / f["value"] if pr.get("value") else None}


def run_extras(args):
    import copy

    import torch

    out = {}
    for key, name, steps in EXTRAS:
        sub_args = copy.copy(args)
        sub_args.workload, sub_args.steps = name, steps
        wl = WORKLOADS[name]
        ln = run_ours(sub_args, wl, sub=True)
        roof = ln["roofline"]
        d = {"workload": name, "value": ln["value"], "unit": ln["unit"], "steps": steps,
             "ms_per_step": ln["ms_per_step"], "e2e": ln["e2e"], "status": ln["status"],
             "roofline": {k: roof[k] for k in ("bound", "achieved", "peak", "unit", "frac", "peak_source")
                          if k in roof},
             "vs_oracle": ln.get("vs_oracle"), "clocks": ln["clocks"]}
        if "other" in roof:
            d["roofline"]["other"] = roof["other"]
        if "vs_squaring" in ln:
            vq = dict(ln["vs_squaring"])
            vq["bar"] = 0.95 * vq["formula_ratio"]  # wall-time target: 0.95 x the product-count ratio
            d["vs_squaring"] = vq
        if "vs_per_matrix" in ln:
            d["vs_per_matrix"] = ln["vs_per_matrix"]
            d["graph_replay"] = ln.get("graph_replay")
            d["resident_matrices"] = ln["config"].get("resident_matrices")
        out[key] = d
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: the workload's, a timed region of about 2 s; 10 for --impl reference)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="time the default launch configuration")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison evaluation")
    ap.add_argument("--launch", type=lambda v: tuple(int(x) for x in v.split(",")), default=None,
                    metavar="PAIR,GROUP",
                    help="split single workloads: set the tile pair (-1/0/1) and raster group by hand")
    ap.add_argument("--fp64-large", action="store_true", help="run the FP64 comparison on the n = 16384 workload")
    ap.add_argument("--no-resident", action="store_true",
                    help="batched workloads: every matrix through the grouped launches (no resident launch)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the secondary workloads (radix 9, precise, batched, FP32)")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.steps is None:
        args.steps = 10 if args.impl == "reference" else wl.get("steps", 10)
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
