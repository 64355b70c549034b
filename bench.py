#!/usr/bin/env python
"""Benchmark: GPSS solves per second to a relative objective gap of 1e-6.

Workload (one step = one full solve of eq. 2 from x0 = 0 until
(f(x) - f*)/f* <= 1e-6): the compressed-sensing instance K 4096 x 16384 FP32,
K iid N(0, 1/4096), 400-sparse Bernoulli-Gaussian x_true, noise 0.01,
rho = 0.9 ||x_true||_1 (seeded synthetic data).  f* is the FP64 oracle's
optimum stored in tests/golden/fstar.json.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).  `value` is device-timed with inputs resident in
HBM; `e2e` repeats the measurement through the public API with the inputs in
pinned host memory (host-to-device copy of K and y and the device-to-host read
of x inside every step).  The solve runs on the library's default engine, the
one-read kernel, whose algorithmic HBM traffic is one read of K per pass (one
pass per iteration plus the setup pass that forms g_0); `roofline` compares
those bytes per launch with the kernel's event-timed duration.  `two_pass`
times the same solves on the two-pass kernel (two reads of K per iteration).
`cpu_baseline` times the FP64 oracle on this host's cores on whole solves of
the same workload.  `--impl reference` runs only that oracle arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "solves/sec to rel. objective gap 1e-6 (batched+warm vs plain GP); HBM GB/s"
TOL = 1e-6


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def golden(name):
    with open(os.path.join(ROOT, "tests", "golden", "fstar.json")) as fh:
        return json.load(fh)[name]


def workload():
    import workloads as W
    return W.config1()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def mark(self, start: bool):
        """Wall-clock bounds of the timed region (samples outside it are ignored)."""
        if start:
            self.t0 = time.monotonic()
        else:
            self.t1 = time.monotonic()

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = getattr(self, "t0", None), getattr(self, "t1", None)
        # nvidia-smi reports each sample a little after taking it: keep the
        # samples that arrive inside the region or within one period after it
        picked = [ln for t, ln in self.lines if t0 is None or (t0 <= t <= t1 + 0.1)]
        for ln in picked:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "interval_ms": 50}


# -------------------------------------------------------------- CPU oracle
def oracle_solve_seconds(prob, fstar, budget_s):
    """Time whole oracle solves of `prob` to the 1e-6 gap; at least one, until budget_s."""
    import oracle
    times, iters = [], []
    while not times or (sum(times) < budget_s and len(times) < 50):
        t0 = time.perf_counter()
        x, res, _ = oracle.gpss(prob, f_star=fstar, tol=TOL)
        times.append(time.perf_counter() - t0)
        iters.append(res.iters)
    return times, iters, oracle.num_threads()


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    prob = workload()
    gold = golden("c1")
    import oracle
    for _ in range(args.warmup):
        oracle.gpss(prob, f_star=gold["f_star"], tol=TOL)
    times, iters, cores = [], [], oracle.num_threads()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, res, _ = oracle.gpss(prob, f_star=gold["f_star"], tol=TOL)
        times.append(time.perf_counter() - t0)
        iters.append(res.iters)
    total = sum(times)
    value = args.steps / total
    sample = f"{args.steps} full oracle solves of {prob.name} to rel gap {TOL:g} ({statistics.mean(iters):.0f} iterations each)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": prob.name, "n": prob.n, "p": prob.p, "stop": f"rel_gap<={TOL:g} vs oracle f*"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------- multi-rank helpers
def max_over_ranks(value_ms: float, world: int, device=None) -> float:
    """The slowest rank's time: every rank passes its own, every rank gets the max."""
    if world <= 1:
        return float(value_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([value_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, max_total_ms: float) -> float:
    """Solves per second of the whole job: every rank solved `steps` instances (weak scaling)."""
    return world * steps / (max_total_ms / 1e3)


def lpt_partition(costs, world: int):
    """Instances to ranks by longest processing time first: in decreasing cost,
    each instance goes to the rank with the least work so far (ties to the
    lower rank).  Every rank computes the same partition from the same costs."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += costs[i]
    return parts


def objective_f64(prob, x) -> float:
    """f(x) = ||K x - y||^2 in FP64 on the stored K (numpy; a check of the returned
    x against the stored optimum, outside every timed region)."""
    import workloads as W
    K = prob.K[:, :prob.p]
    K64 = W.bf16_bits_to_f64(K) if prob.dtype == W.DT_BF16 else np.asarray(K, np.float64)
    r = K64 @ np.asarray(x, np.float64) - np.asarray(prob.y, np.float64)
    return float(r @ r)


# ------------------------------------------------- batched ragged form (c3a)
def run_batched(count, steps, dev, plain_sample=64):
    """Solves/s of `count` instances of the ragged recipe (n in [128, 2048], p = 4n,
    BF16 K, +-1 signals): one persistent gpl1_solve_batched launch per step, the same
    launch replayed from its CUDA graph (gpl1_plan_run), and a sample of the instances
    (every count/plain_sample-th) solved one after another with gpl1_solve (the plain
    form).  Each instance stops at relative gap 1e-6 against the oracle's optimum of
    that instance (tests/golden/c3a_fstar.json, written by tests/golden/make_golden.py)."""
    import torch

    import paper_0902_4424_gb300 as pkg
    import workloads as W
    sizes = W.ragged_sizes(512)[:count]
    probs = [W.ragged_instance(i, n) for i, n in enumerate(sizes)]
    with open(os.path.join(ROOT, "tests", "golden", "c3a_fstar.json")) as fh:
        fstars = json.load(fh)["f_star"][:count]
    keep, descs = [], []
    for pr, fs in zip(probs, fstars):
        K = torch.from_numpy(pr.K.view(np.int16)).to(dev)
        y = torch.from_numpy(pr.y).to(dev)
        x = torch.zeros(pr.p, dtype=torch.float32, device=dev)
        keep.append((K, y, x))
        descs.append(pkg.Context.make_problem(K, y, pr.rho, x, pr.p, fs))
    ctx = pkg.Context(dev.index or 0)
    # the kernel decides on its own (float) estimate of f: stop at half the target
    # so that the gap the oracle verifies on the returned x stays within 1e-6
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=0.5 * TOL, x0_is_zero=1, max_iter=20000)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        ctx.solve_batched(descs, pkg.BF16, prm)
    torch.cuda.synchronize()
    ms, kms, res = [], [], None
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res = ctx.solve_batched(descs, pkg.BF16, prm)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
        kms.append(res[0].kernel_ms)
    ok = sum(r.status == 0 for r in res)
    iters = [r.iters for r in res]
    algo = sum(it * 2.0 * pr.n * pr.p * 2 for it, pr in zip(iters, probs))
    # the same batched solve as a CUDA graph (no host work per replay)
    plan = ctx.plan_batched(descs, pkg.BF16, prm)
    plan.run()
    torch.cuda.synchronize()
    gms = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.run()
        b.record(stream)
        b.synchronize()
        gms.append(a.elapsed_time(b))
    plan.close()
    # the plain form on a sample: one instance after another, each its own cooperative launch
    pick = list(range(0, count, max(1, count // plain_sample)))[:plain_sample]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    plain_ok = 0
    for q in pick:
        K, y, x = keep[q]
        _, r = ctx.solve(K, y, probs[q].rho, x=x, p=probs[q].p, params=prm, f_star=fstars[q])
        plain_ok += r.status == 0
    b.record(stream)
    b.synchronize()
    plain_ms = a.elapsed_time(b) * count / len(pick)   # the whole set at the sample's rate
    # untimed: the oracle's optimum on a few instances, against the batched x
    ctx.solve_batched(descs, pkg.BF16, prm)
    torch.cuda.synchronize()
    gaps = [(objective_f64(probs[q], keep[q][2].double().cpu().numpy()) - fstars[q]) / max(fstars[q], 1e-300)
            for q in range(count)]
    peak, _ = peaks()
    mean_ms = statistics.mean(ms)
    out = {"workload": f"c3a_ragged{count}_bf16", "instances": count, "solves_per_s": count / (mean_ms / 1e3),
           "ms_per_batch": mean_ms, "ok": ok, "iters_mean": statistics.mean(iters), "iters_max": max(iters),
           "graph_solves_per_s": count / (statistics.mean(gms) / 1e3),
           "plain_solves_per_s": count / (plain_ms / 1e3), "plain_sample": len(pick), "plain_ok": plain_ok,
           "speedup_vs_plain": plain_ms / mean_ms, "stop": f"kernel stop rel_gap<={0.5 * TOL:g} vs oracle f* per instance",
           "verified_max_rel_gap": max(gaps) if gaps else None, "verified_instances": len(gaps),
           "hbm_gbs": algo / (statistics.mean(kms) / 1e3) / 1e9}
    out["roofline_frac"] = out["hbm_gbs"] / peak
    # the box shape the batched autotuner chose for this batch (its 4-iteration
    # timings) and, for comparison, the whole batched solve with each shape pinned
    names = {pkg.TILE_SMALL: "small_15KiB", pkg.TILE_MEDIUM: "medium_30KiB", pkg.TILE_LARGE: "large_60KiB"}
    tuned = [t for t in ctx.batched_tuned() if t["key"][1] == count]
    if tuned:
        out["tile_tuned"] = {"choice": names[tuned[0]["tile"]],
                             "tuning_ms": {names[k]: round(v, 4) for k, v in
                                           zip((pkg.TILE_SMALL, pkg.TILE_MEDIUM, pkg.TILE_LARGE), tuned[0]["ms"])}}
    pinned = {}
    for tl, nm in names.items():
        q = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=0.5 * TOL, x0_is_zero=1, max_iter=20000, tile=tl)
        ctx.solve_batched(descs, pkg.BF16, q)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rr = ctx.solve_batched(descs, pkg.BF16, q)
        b.record(stream)
        b.synchronize()
        pinned[nm] = {"ms_per_batch": round(a.elapsed_time(b), 3), "ok": sum(r.status == 0 for r in rr)}
    out["tile_pinned"] = pinned
    ctx.close()
    return out


def run_batched_sharded(rank, world, steps, warmup, dev, count=512):
    """The 512 ragged instances shared out over the ranks by LPT on n p (no
    collective on the data path: each rank solves its share with one batched
    launch per step); the whole job's rate is count instances per step over the
    slowest rank's time (total work fixed: strong scaling).  Rank 0 prints."""
    import torch
    if world > 1:
        import torch.distributed as dist

    import paper_0902_4424_gb300 as pkg
    import workloads as W
    sizes = W.ragged_sizes(512)[:count]
    share = lpt_partition([4.0 * n * n for n in sizes], world)[rank]
    with open(os.path.join(ROOT, "tests", "golden", "c3a_fstar.json")) as fh:
        fstars = json.load(fh)["f_star"][:count]
    probs, keep, descs = [], [], []
    for i in share:
        pr = W.ragged_instance(i, sizes[i])
        K = torch.from_numpy(pr.K.view(np.int16)).to(dev)
        y = torch.from_numpy(pr.y).to(dev)
        x = torch.zeros(pr.p, dtype=torch.float32, device=dev)
        probs.append(pr)
        keep.append((K, y, x))
        descs.append(pkg.Context.make_problem(K, y, pr.rho, x, pr.p, fstars[i]))
    ctx = pkg.Context(dev.index or 0)
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=0.5 * TOL, x0_is_zero=1, max_iter=20000)
    for _ in range(warmup):
        ctx.solve_batched(descs, pkg.BF16, prm)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    a.record(stream)
    ok = 0
    for _ in range(steps):
        res = ctx.solve_batched(descs, pkg.BF16, prm)
        ok = sum(r.status == 0 for r in res)
    b.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    mine = a.elapsed_time(b)
    mx = max_over_ranks(mine, world, dev)
    gaps = [(objective_f64(pr, k[2].double().cpu().numpy()) - fstars[i]) / fstars[i]
            for pr, k, i in list(zip(probs, keep, share))[:8]]
    worst = max_over_ranks(max(gaps) if gaps else 0.0, world, dev)
    ok_all = max_over_ranks(float(len(share) - ok), world, dev)   # the most instances any rank left unsolved
    value = count * steps / (mx / 1e3)
    if rank == 0:
        loads = [sum(4.0 * sizes[i] ** 2 for i in part) for part in lpt_partition([4.0 * n * n for n in sizes], world)]
        print(json.dumps({"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": steps,
                          "warmup": warmup, "ms_per_step": mx / steps, "higher_is_better": True, "scaling": "strong",
                          "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
                          "config": {"workload": f"c3a_ragged{count}_bf16", "parallelism": f"lpt over {world} ranks",
                                     "l2": "each step solves every instance of the share from x0 = 0"},
                          "shares": [len(p) for p in lpt_partition([4.0 * n * n for n in sizes], world)],
                          "load_imbalance": max(loads) / (sum(loads) / world),
                          "unsolved_max_per_rank": ok_all, "verified_max_rel_gap": worst,
                          "gpu_launches": steps}), flush=True)
    ctx.close()


# ------------------------------------------------ shared-K form (c3b)
def run_shared_k(nrhs, dev, verify=16, plain=8, pin=None):
    """Solves/s of nrhs right-hand sides on one K 2048 x 8192 BF16 (each from its own
    +-1 102-sparse signal), all in one gpl1_solve_shared_k call (tensor-core GEMMs),
    against the same instances solved one by one with gpl1_solve (plain form, a
    sample).  Stops at relative gap 5e-7 against the oracle's optimum of each
    instance (tests/golden/c3b_fstar.json); x is checked by the oracle on a sample."""
    import torch

    import paper_0902_4424_gb300 as pkg
    import workloads as W
    with open(os.path.join(ROOT, "tests", "golden", "c3b_fstar.json")) as fh:
        fstars = json.load(fh)["f_star"]
    Ks, ldk, Y, rho, Xt = W.shared_k(nrhs=len(fstars))
    Ks, Y, rho, Xt, fstars = Ks, Y[:nrhs], rho[:nrhs], Xt[:nrhs], fstars[:nrhs]
    n, p = Ks.shape[0], Xt.shape[1]
    K = torch.from_numpy(Ks.view(np.int16)).to(dev)
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).to(dev)
    ctx = pkg.Context(dev.index or 0)
    if pin:   # "cfg:1,cfg:splits": pinned choices for K^T R and K D instead of tuning
        (c1, s1), (c2, s2) = [tuple(int(v) for v in t.split(":")) for t in pin.split(",")]
        ctx.gemm_tuned_set((p, nrhs, 3 * n, n, 1), c1, s1)
        ctx.gemm_tuned_set((n, nrhs, 3 * p, p, 8), c2, s2)
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=0.5 * TOL, max_iter=2000)
    ctx.solve_shared_k(K, Yd, rho, p=p, f_star=fstars, params=prm)          # warm-up
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    X, res = ctx.solve_shared_k(K, Yd, rho, p=p, f_star=fstars, params=prm)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    iters = [r.iters for r in res]
    ok = sum(r.status == 0 for r in res)
    Xh = X.double().cpu().numpy()
    probs = [W.Problem(Ks, n, p, ldk, W.DT_BF16, Y[q].copy(), float(rho[q]), Xt[q], f"c3b_{q}") for q in range(nrhs)]
    idx = np.linspace(0, nrhs - 1, min(verify, nrhs)).astype(int)
    gaps = [(objective_f64(probs[q], Xh[q]) - fstars[q]) / fstars[q] for q in idx]
    # the plain form on a sample: each instance its own cooperative solve of K
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for q in range(plain):
        ctx.solve(K, Yd[q], float(rho[q]), p=p, f_star=fstars[q], params=prm)
    t1.record(stream)
    t1.synchronize()
    plain_ms = t0.elapsed_time(t1) / plain
    # executed tensor-core work: per iteration 2 p nrhs 3n (K^T R) + 2 n nrhs 3p (K D)
    flops = 12.0 * n * p * nrhs * max(iters)
    method_flops = 4.0 * n * p * sum(iters)
    tuned = [{"shape_MNKdKa": list(t["shape"][:4]), "config": t["config"], "splits": t["splits"],
              "ms": round(t["ms"], 4)} for t in ctx.gemm_tuned()]
    peaks_d = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks_d = json.load(fh)
    except OSError:
        pass
    tf_peak = float(peaks_d.get("bf16_tflops", 1900.0))
    out = {"workload": f"c3b_sharedK{n}x{p}_bf16_{nrhs}rhs", "instances": nrhs,
           "solves_per_s": nrhs / (ms / 1e3), "ms_per_call": ms, "ok": ok,
           "iters_mean": statistics.mean(iters), "iters_max": max(iters),
           "plain_solves_per_s": 1e3 / plain_ms, "plain_sample": plain,
           "speedup_vs_plain": (nrhs / (ms / 1e3)) / (1e3 / plain_ms),
           "stop": f"kernel stop rel_gap<={0.5 * TOL:g} vs oracle f* per instance",
           "verified_max_rel_gap": max(gaps), "verified_instances": len(gaps),
           "tensor_tflops": flops / (ms / 1e3) / 1e12,
           "tensor_frac_of_measured_bf16": flops / (ms / 1e3) / 1e12 / tf_peak,
           # the method's own products (2 n p for K^T r, 2 n p for K d, per
           # instance and iteration it ran), without the split of the vector operand
           "method_tflops": method_flops / (ms / 1e3) / 1e12,
           "method_frac_of_measured_bf16": method_flops / (ms / 1e3) / 1e12 / tf_peak,
           "ms_per_iteration": ms / max(iters),
           "gemm_autotuned": tuned,
           "note": "executed GEMM work incl. the 3-term BF16 split of the vector operand; all iterations of the call"}
    ctx.close()
    return out


# ------------------------------------------------ learned warm start (c4)
def run_warm_start(dev, steps=3000, batch=256, lr=3e-4, plain_sample=512, verify=64):
    """The learned warm start at its full configuration (K 1024 x 4096 BF16): 10^5
    training right-hand sides (workloads.warm_start_train) with the solver's own
    solutions as targets (shared-K form, 120 iterations), the network initialised by
    gpl1_lista_init (6 layers, W_l = K^T / L, theta_l = median lambda / L) and
    trained with Adam on the GPU (gpl1_lista_train), then the 10^4 test right-hand
    sides (workloads.warm_start_test) solved to relative gap 1e-6 (kernel stop 5e-7
    against the oracle's optima, tests/golden/c4full_fstar.json) three ways: plain
    (one gpl1_solve per instance, timed on a sample), batched cold (shared-K form
    from x0 = 0) and batched warm (gpl1_solve_warm: inference, warm solve, and the
    cold fallback for any instance the warm solve leaves unconverged).  A spread
    sample of the returned x is checked in FP64."""
    import torch

    import paper_0902_4424_gb300 as pkg
    import workloads as W
    with open(os.path.join(ROOT, "tests", "golden", "c4full_fstar.json")) as fh:
        fstars = json.load(fh)["f_star"]
    Ks, ldk = W.warm_start_K()
    n, p = Ks.shape[0], 4096
    Ytr, rho_tr = W.warm_start_train(W.WARM_TRAIN_FULL, n, p)
    Yte, rho_te = W.warm_start_test(W.WARM_TEST_FULL, n, p)
    ntr, nte = Ytr.shape[0], Yte.shape[0]
    K = torch.from_numpy(Ks.view(np.int16)).to(dev)
    Ytr_d = torch.from_numpy(Ytr).to(dev)
    Yte_d = torch.from_numpy(Yte).to(dev)
    ctx = pkg.Context(dev.index or 0)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731
    chunk = 4096

    def timed(fn):
        a, b = ev(), ev()
        a.record(stream)
        out = fn()
        b.record(stream)
        b.synchronize()
        return out, a.elapsed_time(b)

    # training targets: solutions of eq. 2 for the training samples (shared-K form)
    def targets():
        xs, lams = [], []
        for c0 in range(0, ntr, chunk):
            Xs, res = ctx.solve_shared_k(K, Ytr_d[c0:c0 + chunk], rho_tr[c0:c0 + chunk], p=p,
                                         params=pkg.params_default(stop_rule=0, max_iter=120))
            xs.append(Xs)
            lams += [r.lambda_ for r in res]
        return torch.cat(xs), lams
    (Xtr, lams), target_ms = timed(targets)
    layers = 6
    (Wd, thd, Lk), init_ms = timed(lambda: ctx.lista_init(K, layers, lams, p=p))
    m = torch.zeros(layers * p * n + layers, dtype=torch.float32, device=dev)
    v = torch.zeros_like(m)
    losses, train_ms = timed(lambda: ctx.lista_train(K, Wd, thd, m, v, Ytr_d, Xtr, batch=batch, steps=steps, lr=lr,
                                                     lr_theta=lr))
    del Xtr
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=0.5 * TOL, max_iter=5000)

    def cold():
        xs, rs = [], []
        for c0 in range(0, nte, chunk):
            Xc, rc = ctx.solve_shared_k(K, Yte_d[c0:c0 + chunk], rho_te[c0:c0 + chunk], p=p,
                                        f_star=fstars[c0:c0 + chunk], params=prm)
            xs.append(Xc)
            rs += rc
        return torch.cat(xs), rs
    cold()   # warm-up and GEMM tuning
    (Xc, rc), cold_ms = timed(cold)
    warm = lambda: ctx.solve_warm(K, Wd, thd, Yte_d, rho_te, f_star=fstars, params=prm)   # noqa: E731
    warm()
    (Xw, rw, fb, nfb), warm_ms = timed(warm)
    # plain: one gpl1_solve per instance, on a spread sample
    idx = np.linspace(0, nte - 1, plain_sample).astype(int)
    x1 = torch.zeros(p, dtype=torch.float32, device=dev)

    def plain():
        its = []
        for q in idx:
            _, r = ctx.solve(K, Yte_d[q], float(rho_te[q]), x=x1, p=p,
                             params=pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=0.5 * TOL,
                                                       f_star=fstars[q], x0_is_zero=1, max_iter=5000))
            its.append(r.iters)
        return its
    plain()
    plain_its, plain_ms = timed(plain)
    # the network's output against the cold solutions, and the FP64 check of a sample
    Xn = ctx.lista_forward(K, Wd, thd, Yte_d[:4096])
    test_rel_err = float((((Xn - Xc[:4096]) ** 2).sum(1).mean() / (Xc[:4096] ** 2).sum(1).mean()).sqrt().item())
    vidx = np.linspace(0, nte - 1, verify).astype(int)
    Xwh = Xw[vidx].double().cpu().numpy()
    gaps = []
    for j, q in enumerate(vidx):
        pr = W.Problem(Ks, n, p, ldk, W.DT_BF16, Yte[q].copy(), float(rho_te[q]), None, "c4")
        gaps.append((objective_f64(pr, Xwh[j]) - fstars[q]) / fstars[q])
    ctx.close()
    return {"workload": f"c4_warmstart{n}x{p}_bf16", "train_samples": ntr, "test_samples": nte,
            "layers": layers, "train_steps": steps, "batch": batch, "spectral_norm_sq": Lk,
            "target_solve_ms": target_ms, "init_ms": init_ms, "train_ms": train_ms,
            "loss_first": float(np.mean(losses[:8])), "loss_last": float(np.mean(losses[-8:])),
            "test_rel_err": test_rel_err,
            "plain_solves_per_s": len(idx) / (plain_ms / 1e3), "plain_iters_mean": statistics.mean(plain_its),
            "plain_sample": len(idx),
            "cold_solves_per_s": nte / (cold_ms / 1e3), "warm_solves_per_s": nte / (warm_ms / 1e3),
            "cold_iters_mean": statistics.mean(r.iters for r in rc),
            "warm_iters_mean": statistics.mean(r.iters for r in rw),
            "cold_ok": sum(r.status == 0 for r in rc), "warm_ok": sum(r.status == 0 for r in rw),
            "fallbacks": nfb, "warm_verified_max_rel_gap": max(gaps), "verified_instances": len(gaps),
            "stop": f"kernel stop rel_gap<={0.5 * TOL:g} vs oracle f* per test sample",
            "note": "warm time includes the network's inference and the cold fallbacks; batched forms in "
                    "shared-K calls of 4096 right-hand sides"}


# ------------------------------------------------ radius sweep (c5)
def run_rho_sweep(dev):
    """The paper's Gaussian shape (K 1848 x 8192, ||K|| = 1, 2% noise; rows padded to
    1856) solved for 50 radii from 0.05 to 1.2 ||x_true||_1 (workloads.rho_sweep):
    (a) all radii in one gpl1_solve_shared_k call, (b) one gpl1_solve per radius in
    increasing order, each started from the previous solution (continuation along
    rho), (c) one cold gpl1_solve per radius.  Each stops at relative gap 5e-7
    against the oracle's optimum of that radius (tests/golden/c5_fstar.json), the
    gap taken relative to max(f*, 1e-6 ||y||^2) (f* is tiny once rho allows a
    near-exact fit); every returned x is checked in FP64."""
    import torch

    import paper_0902_4424_gb300 as pkg
    import workloads as W
    with open(os.path.join(ROOT, "tests", "golden", "c5_fstar.json")) as fh:
        fstars = json.load(fh)["f_star"]
    Ks, ldk, n, y, rho, xt = W.rho_sweep()
    p, R = xt.shape[0], len(rho)
    K = torch.from_numpy(Ks.view(np.int16)).to(dev)
    yd = torch.from_numpy(y).to(dev)
    Yd = yd.unsqueeze(0).repeat(R, 1).contiguous()
    ctx = pkg.Context(dev.index or 0)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=0.5 * TOL, max_iter=20000)
    y2 = float(np.dot(y.astype(np.float64), y.astype(np.float64)))
    den = [max(f, 1e-6 * y2) for f in fstars]
    prob = W.Problem(Ks, n, p, ldk, W.DT_BF16, y.astype(np.float32), 0.0, xt, "c5")

    def gaps(X):
        return [(objective_f64(prob, X[b]) - fstars[b]) / den[b] for b in range(R)]
    ctx.solve_shared_k(K, Yd, rho, p=p, f_star=fstars, params=prm)   # warm-up and tuning
    a, b = ev(), ev()
    a.record(stream)
    Xs, rs = ctx.solve_shared_k(K, Yd, rho, p=p, f_star=fstars, params=prm)
    b.record(stream)
    b.synchronize()
    shared_ms = a.elapsed_time(b)
    g_shared = gaps(Xs.double().cpu().numpy())
    out = {"workload": f"c5_rhosweep1848x8192_bf16_{R}", "radii": R,
           "shared_k": {"solves_per_s": R / (shared_ms / 1e3), "ms": shared_ms,
                        "iters_mean": statistics.mean(r.iters for r in rs), "ok": sum(r.status == 0 for r in rs),
                        "verified_max_rel_gap": max(g_shared)}}
    for mode in ("continuation", "cold"):
        x = torch.zeros(p, dtype=torch.float32, device=dev)
        xs, its, oks = [], [], 0
        a, b = ev(), ev()
        a.record(stream)
        for q in range(R):
            if mode == "cold":
                x = torch.zeros(p, dtype=torch.float32, device=dev)
            x, r = ctx.solve(K, yd, float(rho[q]), x=x, p=p, params=prm, f_star=fstars[q])
            xs.append(x.clone())
            its.append(r.iters)
            oks += r.status == 0
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        g = gaps(torch.stack(xs).double().cpu().numpy())
        out[mode] = {"solves_per_s": R / (ms / 1e3), "ms": ms, "iters_mean": statistics.mean(its), "ok": oks,
                     "verified_max_rel_gap": max(g)}
    # isochrones (Sec. 4): all radii under a fixed iteration budget (no stop rule), the
    # time of the call, and per radius the relative error ||x - x_bar|| / ||x_bar||
    # against the exact point of the homotopy path (tests/golden/xbar_c5.npz) and the gap
    import sys as _sys
    _sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    from make_golden import load_sparse
    xbar = load_sparse(os.path.join(ROOT, "tests", "golden", "xbar_c5.npz"))[0]
    iso = []
    for budget in (4, 8, 16, 32, 64, 128):
        prm_b = pkg.params_default(stop_rule=0, max_iter=budget)
        a, b = ev(), ev()
        a.record(stream)
        Xb, _ = ctx.solve_shared_k(K, Yd, rho, p=p, params=prm_b)
        b.record(stream)
        b.synchronize()
        Xh = Xb.double().cpu().numpy()
        g = gaps(Xh)
        err = [float(np.linalg.norm(Xh[q] - xbar[q]) / np.linalg.norm(xbar[q])) for q in range(R)]
        iso.append({"iterations": budget, "ms": a.elapsed_time(b), "x_err_median": float(np.median(err)),
                    "x_err_max": float(max(err)), "gap_median": float(np.median(g)), "gap_max": float(max(g))})
    out["isochrones"] = iso
    out["stop"] = f"kernel stop gap<={0.5 * TOL:g} vs oracle f* per radius, relative to max(f*, 1e-6 ||y||^2)"
    ctx.close()
    return out


# -------------------------------------------------------------- GPU path
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_0902_4424_gb300 as pkg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pkg.lib()   # the compiled library must be present: no fallback
    prob = workload()
    gold = golden("c1")
    fstar = gold["f_star"]
    n, p = prob.n, prob.p
    K_host = torch.from_numpy(prob.K).pin_memory()
    y_host = torch.from_numpy(prob.y).pin_memory()
    x_host = torch.empty(p, dtype=torch.float32).pin_memory()
    K = K_host.to(dev)
    y = y_host.to(dev)
    x = torch.zeros(p, dtype=torch.float32, device=dev)
    ctx = pkg.Context(local_rank)
    engine = {"one_read": pkg.ENGINE_ONE_READ, "nch2": pkg.ENGINE_ONE_READ_NCH2, "nch4": pkg.ENGINE_ONE_READ_NCH4,
              "two_pass": pkg.ENGINE_TWO_PASS, "auto": pkg.ENGINE_AUTO}[args.engine]
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=TOL, f_star=fstar, x0_is_zero=1, max_iter=20000,
                             engine=engine)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 512 MiB > L2

    def solve():
        xx, res = ctx.solve(K, y, prob.rho, x=x, p=p, params=prm)
        if res.status != 0:
            raise RuntimeError(f"solve failed: {res.as_dict()}")
        return res

    clk = ClockSampler(local_rank).__enter__()   # running before the timed region starts
    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    time.sleep(0.3)

    # ---- device-timed steps (inputs resident in HBM, L2 flushed between steps)
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kernel_ms, iters = [], []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.mark(True)
    for s in range(args.steps):
        flush.fill_(float(s))
        evs[s][0].record(stream)
        res = solve()
        evs[s][1].record(stream)
        kernel_ms.append(res.kernel_ms)
        iters.append(res.iters)
    torch.cuda.synchronize()
    clk.mark(False)
    time.sleep(0.15)
    clk.__exit__(None, None, None)
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    total_ms_max = max_over_ranks(total_ms, world, dev)
    value = whole_job_rate(world, args.steps, total_ms_max)

    # ---- check the objective actually reached (FP64 on the host, untimed)
    f_gpu = objective_f64(prob, x.double().cpu().numpy())
    verified_gap = (f_gpu - fstar) / fstar

    # ---- end to end through the public API with host buffers: every step copies its K
    # and y from pinned host memory and reads x back.  The copies of step s + 1 run on a
    # second stream while step s solves (two device buffers), as a user pipelines them.
    h2d = K_host.numel() * K_host.element_size() + y_host.numel() * y_host.element_size()
    d2h = x_host.numel() * x_host.element_size()
    Kb, yb = [K, torch.empty_like(K)], [y, torch.empty_like(y)]
    copy_stream = torch.cuda.Stream(device=dev)
    ready = [torch.cuda.Event(), torch.cuda.Event()]

    def stage(slot):   # inputs of one step into buffer `slot`, on the copy stream
        with torch.cuda.stream(copy_stream):
            Kb[slot].copy_(K_host, non_blocking=True)
            yb[slot].copy_(y_host, non_blocking=True)
            ready[slot].record(copy_stream)

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    copy_stream.wait_event(a)
    stage(0)
    for s in range(args.steps):
        i = s % 2
        if s + 1 < args.steps:
            stage(1 - i)   # buffer 1 - i served step s - 1, whose solve has returned
        stream.wait_event(ready[i])
        _, res = ctx.solve(Kb[i], yb[i], prob.rho, x=x, p=p, params=prm)
        if res.status != 0:
            raise RuntimeError(f"solve failed: {res.as_dict()}")
        x_host.copy_(x, non_blocking=True)
    b.record(stream)
    b.synchronize()
    e2e_value = whole_job_rate(world, args.steps, max_over_ranks(a.elapsed_time(b), world, dev))

    if rank != 0:
        return
    # ---- roofline of the solver kernel: one read of K per pass, one pass per
    # iteration plus the setup pass
    bytes_per_pass = 1.0 * n * p * prob.K.itemsize
    mean_iters = statistics.mean(iters)
    algo_bytes = bytes_per_pass * (mean_iters + 1)
    kms = statistics.mean(kernel_ms)
    achieved = algo_bytes / (kms / 1e3) / 1e9
    peak, peak_kind = peaks()
    # the kernel that ran the timed solves: the autotuner's choice for this shape,
    # or the engine pinned on the command line
    labels = {pkg.ENGINE_ONE_READ_NCH2: "gpl1::fz::fused_kernel<1,2> (one-read engine, two column chunks per thread)",
              pkg.ENGINE_ONE_READ_NCH4: "gpl1::fz::fused_kernel<1,4> (one-read engine, four column chunks per thread)",
              pkg.ENGINE_TWO_PASS: "gpl1::gpss_kernel<1,2> (two-pass engine)"}
    ran = engine
    for t in ctx.solve_tuned():
        if t["shape"][1] == n and t["shape"][2] == p and engine in (pkg.ENGINE_AUTO, pkg.ENGINE_ONE_READ):
            ran = t["engine"]
    kernel_label = labels.get(ran, str(ran))
    traffic = None
    tr_file = os.path.join(ROOT, "profiles", "fused_kernel_c1_f32_traffic.txt")   # JSON text
    if os.path.exists(tr_file):
        with open(tr_file) as fh:
            tr = json.load(fh)
        if (tr.get("workload") == prob.name and tr.get("kernel_fingerprint") == kernel_fingerprint()
                and kernel_label.startswith(tr.get("kernel", "?"))):
            traffic = tr.get("dram_bytes_per_launch")

    # ---- CPU baseline: the oracle on this host's cores, one bounded sample
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        times, oit, cores = oracle_solve_seconds(prob, fstar, budget_s=args.cpu_budget)
        cpu = {"value": len(times) / sum(times), "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": f"{len(times)} full FP64 oracle solve(s) of {prob.name} to rel gap {TOL:g} "
                         f"({statistics.mean(oit):.0f} iterations each), {sum(times):.1f} s"}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": prob.name, "n": n, "p": p, "rho": prob.rho, "stop": f"rel_gap<={TOL:g} vs oracle f*",
                   "engine": args.engine,
                   "x0": "zero", "l2": "K (256 MiB) exceeds L2; 512 MiB flush between steps",
                   "parallelism": "replicas" if world > 1 else "single"},
        "iters_per_solve": mean_iters,
        "iters_per_s": mean_iters * value / world,
        "time_to_tol_ms": total_ms_max / args.steps,
        "hbm_gbs": achieved,
        "verified_rel_gap": verified_gap,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind,
                     "frac_of_nominal_8tbs": achieved / 8000.0,
                     "kernel": kernel_label,
                     "algorithmic_bytes_per_launch": algo_bytes,
                     "algorithmic_bytes": "one read of K (n p 4 B) per pass; passes = iterations + 1",
                     "kernel_ms": kms},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
    }
    if args.extras:
        line["two_pass"] = run_engine_compare(ctx, K, y, prob, prm, flush, args.steps, dev)
        line["fw_stop"] = run_fw_stop(ctx, K, y, prob, fstar, flush, args.steps, dev)
        line["methods"] = run_methods(ctx, K, y, prob, flush, min(args.steps, 5), dev)
        line["c0"] = run_small_config("c0", dev, 20)
        line["c2"] = run_small_config("c2", dev, 10)
    if args.batched_sample > 0:
        line["batched"] = run_batched(args.batched_sample, 3, dev)
    if args.shared_k > 0 and os.path.exists(os.path.join(ROOT, "tests", "golden", "c3b_fstar.json")):
        line["shared_k"] = run_shared_k(args.shared_k, dev, pin=args.shared_k_pin)
    if args.warm_start and os.path.exists(os.path.join(ROOT, "tests", "golden", "c4full_fstar.json")):
        line["warm_start"] = run_warm_start(dev)
    if args.rho_sweep and os.path.exists(os.path.join(ROOT, "tests", "golden", "c5_fstar.json")):
        line["rho_sweep"] = run_rho_sweep(dev)
    print(json.dumps(line), flush=True)
    ctx.close()


def timed_solves(ctx, K, y, prob, prm, flush, steps, dev):
    """Device time (ms per solve) and results of `steps` solves, L2 flushed before each."""
    import torch
    stream = torch.cuda.current_stream()
    x = torch.zeros(prob.p, dtype=torch.float64 if K.dtype == torch.float64 else torch.float32, device=dev)
    ms, res = [], []
    for s in range(steps):
        flush.fill_(float(s))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, r = ctx.solve(K, y, prob.rho, x=x, p=prob.p, params=prm)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
        res.append(r)
    return ms, res


def run_engine_compare(ctx, K, y, prob, prm, flush, steps, dev):
    """The same solves (c1, stop at the 1e-6 gap) on the two-pass kernel, which
    reads K twice per iteration (K^T r, then [K d, K x]); its roofline counts
    those two reads."""
    import paper_0902_4424_gb300 as pkg
    prm2 = pkg.Params.from_buffer_copy(prm)
    prm2.engine = pkg.ENGINE_TWO_PASS
    timed_solves(ctx, K, y, prob, prm2, flush, 2, dev)
    ms, res = timed_solves(ctx, K, y, prob, prm2, flush, steps, dev)
    iters = statistics.mean(r.iters for r in res)
    kms = statistics.mean(r.kernel_ms for r in res)
    algo = 2.0 * prob.n * prob.p * prob.K.itemsize * iters
    peak, _ = peaks()
    return {"kernel": "gpl1::gpss_kernel<1,2> (two-pass engine, 30 KiB boxes)", "solves_per_s": 1e3 / statistics.mean(ms),
            "ms_per_solve": statistics.mean(ms), "iters_per_solve": iters, "kernel_ms": kms,
            "hbm_gbs": algo / (kms / 1e3) / 1e9, "roofline_frac": algo / (kms / 1e3) / 1e9 / peak,
            "algorithmic_bytes": "two reads of K per iteration", "ok": sum(r.status == 0 for r in res)}


def run_fw_stop(ctx, K, y, prob, fstar, flush, steps, dev):
    """Time to tolerance as a user without f* gets it: the stop on the Frank-Wolfe
    certificate g^T x + rho ||g||_inf <= tol (f - cert) (an upper bound of the
    relative gap), at the tolerances an FP32 gradient can certify on this
    instance (the certificate cancels two terms of size rho ||g||_inf, about 70 f
    here, so FP32 rounding of g bounds what it resolves near 1e-6); the returned
    x's gap checked in FP64."""
    import torch

    import paper_0902_4424_gb300 as pkg
    out = {"stop": "FW certificate <= tol (f - cert), no f*"}
    for tol in (1e-4, 1e-5):
        prm = pkg.params_default(stop_rule=pkg.STOP_ON_FW, tol=tol, x0_is_zero=1, max_iter=2000,
                                 engine=pkg.ENGINE_ONE_READ)   # x0 = 0 (x0_is_zero) in every solve
        timed_solves(ctx, K, y, prob, prm, flush, 1, dev)
        ms, res = timed_solves(ctx, K, y, prob, prm, flush, min(steps, 10), dev)
        x, r = ctx.solve(K, y, prob.rho, p=prob.p, params=prm)
        torch.cuda.synchronize()
        gap = (objective_f64(prob, x.double().cpu().numpy()) - fstar) / fstar
        out[f"tol_{tol:g}"] = {"solves_per_s": 1e3 / statistics.mean(ms), "ms_per_solve": statistics.mean(ms),
                               "iters_per_solve": statistics.mean(r.iters for r in res),
                               "stop_reasons": sorted({pkg.STOP[r.stop] for r in res}),
                               "verified_rel_gap": gap, "ok": sum(r.status == 0 for r in res)}
    return out


def run_methods(ctx, K, y, prob, flush, steps, dev):
    """The comparison methods of Sec. 2 on the same kernel and workload (c1), next to
    Alg. GP + SS: ISTA and FISTA on eq. 1 at the lambda of the lambda-rho relation
    (stored with f*) with step 1/||K||^2 (gpl1_spectral_norm_sq, timed apart), and
    PSD on eq. 2.  Each stops at the distance to its optimum the GPSS solve stops
    at, ||K (x - x*)||^2 <= 5e-7 f*: relative gap 5e-7 in f for GPSS and PSD, the
    same absolute gap in eq. 1's objective (optimum f* + 2 lambda rho) for ISTA and
    FISTA.  Reported per method: solves/s, iterations, passes over K (PSD takes two
    per iteration) and the x error against the oracle's x*."""
    import sys as _sys

    import torch

    import paper_0902_4424_gb300 as pkg
    _sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    from make_golden import load_sparse
    gold = golden("c1")
    lam, fs = gold["lambda"], gold["f_star"]
    xs = load_sparse(os.path.join(ROOT, "tests", "golden", "xstar_c1.npz"))[0][0]
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    L = ctx.spectral_norm_sq(K, pkg.F32, p=prob.p, iters=100)
    b.record(stream)
    b.synchronize()
    out = {"workload": prob.name, "lambda": lam, "spectral_norm_sq": L, "spectral_norm_ms": a.elapsed_time(b),
           "stop": "||K(x - x*)||^2 <= 5e-7 f* (rel gap 5e-7 in f; eq. 1: the same absolute gap)"}
    Fs = fs + 2.0 * lam * prob.rho
    for name, method in (("gpss", pkg.METHOD_GPSS), ("ista", pkg.METHOD_ISTA), ("fista", pkg.METHOD_FISTA),
                         ("psd", pkg.METHOD_PSD)):
        if method in (pkg.METHOD_ISTA, pkg.METHOD_FISTA):
            kw = dict(f_star=Fs, tol=5e-7 * fs / Fs, lambda_pen=lam, step=1.0 / L)
        else:
            kw = dict(f_star=fs, tol=5e-7)
        prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, x0_is_zero=1, max_iter=20000, method=method,
                                 engine=pkg.ENGINE_ONE_READ, **kw)
        timed_solves(ctx, K, y, prob, prm, flush, 1, dev)
        ms, res = timed_solves(ctx, K, y, prob, prm, flush, steps, dev)
        x, r = ctx.solve(K, y, prob.rho, p=prob.p, params=prm)
        torch.cuda.synchronize()
        xh = x.double().cpu().numpy()
        iters = statistics.mean(q.iters for q in res)
        out[name] = {"solves_per_s": 1e3 / statistics.mean(ms), "ms_per_solve": statistics.mean(ms),
                     "iters_per_solve": iters,
                     "passes_per_solve": (2 * iters if method == pkg.METHOD_PSD else iters) + 1,
                     "x_rel_err": float(np.linalg.norm(xh - xs) / np.linalg.norm(xs)),
                     "ok": sum(q.status == 0 for q in res)}
    return out


def run_small_config(name, dev, steps):
    """c0 (FP64 256 x 1024: K is 2 MiB, L2-resident, so latency- and barrier-bound:
    microseconds per iteration) and c2 (FP32 4096 x 4096 ill-conditioned: 64 MiB,
    inside L2 between passes, reported as effective GB/s), each on both engines to
    the 1e-6 gap against the stored oracle optimum; c0 also times the oracle
    single-threaded (whole solves)."""
    import torch

    import oracle
    import paper_0902_4424_gb300 as pkg
    import workloads as W
    prob = {"c0": W.config0, "c2": W.config2}[name]()
    fstar = golden(name)["f_star"]
    K = torch.from_numpy(prob.K).to(dev)
    y = torch.from_numpy(prob.y).to(dev)
    ctx = pkg.Context(dev.index or 0)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {"workload": prob.name, "n": prob.n, "p": prob.p}
    for label, engine, reads in (("one_read", pkg.ENGINE_ONE_READ, None), ("two_pass", pkg.ENGINE_TWO_PASS, 2.0)):
        prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=TOL, f_star=fstar, x0_is_zero=1,
                                 max_iter=20000, engine=engine)
        timed_solves(ctx, K, y, prob, prm, flush, 2, dev)
        ms, res = timed_solves(ctx, K, y, prob, prm, flush, steps, dev)
        iters = statistics.mean(r.iters for r in res)
        kms = statistics.mean(r.kernel_ms for r in res)
        byts = (iters + 1 if reads is None else reads * iters) * prob.n * prob.p * prob.K.itemsize
        out[label] = {"solves_per_s": 1e3 / statistics.mean(ms), "iters_per_solve": iters,
                      "us_per_iter": 1e3 * kms / max(iters, 1), "effective_gbs": byts / (kms / 1e3) / 1e9,
                      "ok": sum(r.status == 0 for r in res)}
    if name == "c0":
        oracle.set_threads(1)
        t0 = time.perf_counter()
        _, r, _ = oracle.gpss(prob, f_star=fstar, tol=TOL)
        dt = time.perf_counter() - t0
        oracle.set_threads(0)
        out["oracle_1thread"] = {"us_per_iter": 1e6 * dt / max(r.iters, 1), "iters": r.iters, "cores": 1,
                                 "solves_per_s": 1.0 / dt}
    if name == "c2":
        out["note"] = "K (64 MiB) stays in L2 between passes: effective GB/s, not an HBM roofline"
    ctx.close()
    return out


def kernel_fingerprint():
    """Hash of the code the solver kernel is compiled from (comments and blank
    lines left out); a stored DRAM-traffic figure is only used while it matches."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_0902_4424_gb300", "csrc")
    for name in ("common.cuh", "gpss.cuh", "project.cuh", "fused.cuh", "fused.cu"):
        with open(os.path.join(csrc, name)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        code = [ln.split("//", 1)[0].rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in code if ln).encode())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--engine", choices=["one_read", "nch2", "nch4", "two_pass", "auto"], default="one_read",
                    help="the main solve's engine (one_read: the autotuner picks the chunks per thread; a "
                         "fixed choice for profiling, which distorts the tuner's timings)")
    ap.add_argument("--batched-sample", type=int, default=512,
                    help="also time this many ragged instances batched vs plain (0: skip)")
    ap.add_argument("--shared-k", type=int, default=1024,
                    help="also time this many right-hand sides on one shared K (0: skip)")
    ap.add_argument("--shared-k-pin", default=None,
                    help="pin the shared-K products' GEMM choices instead of tuning: 'cfg:1,cfg:splits' for "
                         "K^T R and K D (to reproduce a configuration under a profiler)")
    ap.add_argument("--warm-start", type=int, default=1, help="also measure the learned warm start (0: skip)")
    ap.add_argument("--rho-sweep", type=int, default=1, help="also measure the 50-radius sweep (0: skip)")
    ap.add_argument("--extras", type=int, default=1,
                    help="also time c1 on the two-pass engine and with the FW stop, and c0 and c2 (0: skip)")
    ap.add_argument("--workload", choices=["c1", "c3a"], default="c1",
                    help="c3a: only the batched ragged form, all 512 instances")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "c3a" and world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        run_batched_sharded(rank, world, max(1, args.steps // 20), max(args.warmup, 3),
                            torch.device("cuda", local_rank))
    elif args.workload == "c3a":
        import torch
        torch.cuda.set_device(local_rank)
        out = run_batched(512, max(1, args.steps // 20), torch.device("cuda", local_rank))
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": out["solves_per_s"], "unit": "solves/s",
                              "n_gpus": world, "steps": max(1, args.steps // 20), "warmup": 2,
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                              "data": "synthetic", "config": {"workload": out["workload"]}, "batched": out}),
                  flush=True)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
