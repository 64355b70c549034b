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


def load_baseline_metric():
    try:
        with open(os.path.join(ROOT, "BASELINE.json")) as fh:
            return json.load(fh).get("metric", METRIC)
    except OSError:
        return METRIC


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
        "impl": "reference", "metric": load_baseline_metric(), "value": value, "unit": "solves/s",
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
    ctx.close()
    return out


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
           "gemm_autotuned": tuned,
           "note": "executed GEMM work incl. the 3-term BF16 split of the vector operand; all iterations of the call"}
    ctx.close()
    return out


# ------------------------------------------------ learned warm start (c4)
def run_warm_start(dev, steps=3000, batch=256, ntrain=65536, lr=3e-4):
    """The learned warm start on K 1024 x 4096 (BF16): `ntrain` training right-hand
    sides (workloads.warm_start_train) with the solver's own solutions as targets
    (shared-K form), the network (6 layers, W_l initialised to K^T / ||K||^2,
    theta_l to the median lambda / ||K||^2) trained with Adam on the GPU, and the
    test samples solved to relative gap 1e-6 (kernel stop 5e-7, stored oracle
    optima) from x0 = 0 (cold) and from the projected network output (warm,
    inference included; alpha_0 from the projected-gradient step at x0, rule 1)."""
    import torch

    import paper_0902_4424_gb300 as pkg
    import workloads as W
    with open(os.path.join(ROOT, "tests", "golden", "c4_fstar.json")) as fh:
        gold = json.load(fh)
    Ks, ldk, Y, rho, Xt, ntr0 = W.warm_start_split()
    n, p = Ks.shape[0], Xt.shape[1]
    nte = Y.shape[0] - ntr0
    fstars = gold["f_star"]
    Ytr, rho_tr = W.warm_start_train(ntrain, n, p)
    K = torch.from_numpy(Ks.view(np.int16)).to(dev)
    # training samples first, then the test samples (the last rows of the split)
    Yd = torch.from_numpy(np.ascontiguousarray(np.concatenate([Ytr, Y[ntr0:]]))).to(dev)
    rho = np.concatenate([rho_tr, rho[ntr0:]])
    ntr = ntrain
    ctx = pkg.Context(dev.index or 0)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731
    # training targets: solutions of eq. 2 for the training samples (shared-K form)
    a, b = ev(), ev()
    a.record(stream)
    targets, lams = [], []
    for c0 in range(0, ntr, 4096):
        Xs, res = ctx.solve_shared_k(K, Yd[c0:c0 + 4096], rho[c0:c0 + 4096], p=p,
                                     params=pkg.params_default(stop_rule=0, max_iter=120))
        targets.append(Xs)
        lams += [r.lambda_ for r in res]
    Xtr = torch.cat(targets)
    b.record(stream)
    b.synchronize()
    target_ms = a.elapsed_time(b)
    # network: W_l = K^T / L, theta_l = median(lambda) / L, L = ||K||_2^2
    K64 = W.bf16_bits_to_f64(Ks[:, :p])
    Lk = float(np.linalg.norm(K64, 2) ** 2)
    layers = 6
    Wd = (torch.from_numpy((K64.T / Lk).astype(np.float32)).to(dev)).unsqueeze(0).repeat(layers, 1, 1).contiguous()
    thd = torch.full((layers,), float(np.median(lams)) / Lk, dtype=torch.float32, device=dev)
    m = torch.zeros(layers * p * n + layers, dtype=torch.float32, device=dev)
    v = torch.zeros_like(m)
    a, b = ev(), ev()
    a.record(stream)
    losses = ctx.lista_train(K, Wd, thd, m, v, Yd[:ntr], Xtr, batch=batch, steps=steps, lr=lr, lr_theta=lr)
    b.record(stream)
    b.synchronize()
    train_ms = a.elapsed_time(b)
    # test: cold and warm solves of the test samples
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=0.5 * TOL, max_iter=5000)
    Yte = Yd[ntr:]
    ctx.solve_shared_k(K, Yte, rho[ntr:], p=p, f_star=fstars, params=prm)   # warm-up
    a, b = ev(), ev()
    a.record(stream)
    Xc, rc = ctx.solve_shared_k(K, Yte, rho[ntr:], p=p, f_star=fstars, params=prm)
    b.record(stream)
    b.synchronize()
    cold_ms = a.elapsed_time(b)
    prm_w = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=0.5 * TOL, max_iter=5000, alpha0_rule=1)
    a, b = ev(), ev()
    a.record(stream)
    X0 = ctx.lista_forward(K, Wd, thd, Yte)
    Xw, rw = ctx.solve_shared_k(K, Yte, rho[ntr:], p=p, f_star=fstars, params=prm_w, X=X0)
    b.record(stream)
    b.synchronize()
    warm_ms = a.elapsed_time(b)
    # the network's output (the solve above overwrote X0) against the solutions, on the test samples
    Xn = ctx.lista_forward(K, Wd, thd, Yte)
    test_rel_err = float((((Xn - Xc) ** 2).sum(1).mean() / (Xc ** 2).sum(1).mean()).sqrt().item())
    probs = [W.Problem(Ks, n, p, ldk, W.DT_BF16, Y[ntr0 + q].copy(), float(rho[ntr + q]), Xt[ntr0 + q], "c4")
             for q in range(nte)]
    Xwh = Xw.double().cpu().numpy()
    idx = np.linspace(0, nte - 1, 16).astype(int)
    gaps = [(objective_f64(probs[q], Xwh[q]) - fstars[q]) / fstars[q] for q in idx]
    ctx.close()
    return {"workload": f"c4_warmstart{n}x{p}_bf16", "train_samples": ntr, "test_samples": nte,
            "layers": layers, "train_steps": steps, "batch": batch, "train_ms": train_ms,
            "target_solve_ms": target_ms, "loss_first": float(np.mean(losses[:8])),
            "loss_last": float(np.mean(losses[-8:])),
            "test_rel_err": test_rel_err,
            "cold_solves_per_s": nte / (cold_ms / 1e3), "warm_solves_per_s": nte / (warm_ms / 1e3),
            "cold_iters_mean": statistics.mean(r.iters for r in rc),
            "warm_iters_mean": statistics.mean(r.iters for r in rw),
            "cold_ok": sum(r.status == 0 for r in rc), "warm_ok": sum(r.status == 0 for r in rw),
            "warm_verified_max_rel_gap": max(gaps), "verified_instances": len(gaps),
            "stop": f"kernel stop rel_gap<={0.5 * TOL:g} vs oracle f* per test sample",
            "note": "warm time includes the network's inference; both solved in one shared-K call"}


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
    # isochrones: all radii under a fixed iteration budget (no stop rule), the time of
    # the call and the gap each radius reached
    iso = []
    for budget in (4, 8, 16, 32):
        prm_b = pkg.params_default(stop_rule=0, max_iter=budget)
        a, b = ev(), ev()
        a.record(stream)
        Xb, _ = ctx.solve_shared_k(K, Yd, rho, p=p, params=prm_b)
        b.record(stream)
        b.synchronize()
        g = gaps(Xb.double().cpu().numpy())
        iso.append({"iterations": budget, "ms": a.elapsed_time(b), "gap_median": float(np.median(g)),
                    "gap_max": float(max(g))})
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
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=TOL, f_star=fstar, x0_is_zero=1, max_iter=20000,
                             engine=pkg.ENGINE_ONE_READ)
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
    traffic = None
    tr_file = os.path.join(ROOT, "profiles", "fused_kernel_c1_f32_traffic.txt")   # JSON text
    if os.path.exists(tr_file):
        with open(tr_file) as fh:
            tr = json.load(fh)
        if tr.get("workload") == prob.name and tr.get("kernel_fingerprint") == kernel_fingerprint():
            traffic = tr.get("dram_bytes_per_launch")

    # ---- CPU baseline: the oracle on this host's cores, one bounded sample
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        times, oit, cores = oracle_solve_seconds(prob, fstar, budget_s=args.cpu_budget)
        cpu = {"value": len(times) / sum(times), "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": f"{len(times)} full FP64 oracle solve(s) of {prob.name} to rel gap {TOL:g} "
                         f"({statistics.mean(oit):.0f} iterations each), {sum(times):.1f} s"}

    line = {
        "metric": load_baseline_metric(), "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": prob.name, "n": n, "p": p, "rho": prob.rho, "stop": f"rel_gap<={TOL:g} vs oracle f*",
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
                     "kernel": "gpl1::fz::fused_kernel<1,1> (one-read engine)",
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
        line["c0"] = run_small_config("c0", dev, 20)
        line["c2"] = run_small_config("c2", dev, 10)
    if args.batched_sample > 0:
        line["batched"] = run_batched(args.batched_sample, 3, dev)
    if args.shared_k > 0 and os.path.exists(os.path.join(ROOT, "tests", "golden", "c3b_fstar.json")):
        line["shared_k"] = run_shared_k(args.shared_k, dev, pin=args.shared_k_pin)
    if args.warm_start and os.path.exists(os.path.join(ROOT, "tests", "golden", "c4_fstar.json")):
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
    return {"kernel": "gpl1::gpss_kernel<1> (two-pass engine)", "solves_per_s": 1e3 / statistics.mean(ms),
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
    """Hash of the sources the solver kernel is compiled from; a stored DRAM-traffic
    figure is only used while it matches."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_0902_4424_gb300", "csrc")
    for name in ("common.cuh", "gpss.cuh", "project.cuh", "fused.cuh", "fused.cu"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
    elif args.workload == "c3a":
        import torch
        torch.cuda.set_device(local_rank)
        out = run_batched(512, max(1, args.steps // 20), torch.device("cuda", local_rank))
        if rank == 0:
            print(json.dumps({"metric": load_baseline_metric(), "value": out["solves_per_s"], "unit": "solves/s",
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
