"""Write tests/golden/fstar.json: optimal objective values of the measured configurations.

Every number here comes from the FP64 oracle (oracle/) run on the seeded
inputs of workloads/ to its precision floor (Frank-Wolfe certificate 1e-13 or
no decrease of f for 30 iterations).  Nothing here touches the CUDA path.

    python tests/golden/make_golden.py [c0 c1 c2 ...]
    python tests/golden/make_golden.py c3a      # the ragged batch: c3a_fstar.json
    python tests/golden/make_golden.py c3b      # the shared-K right-hand sides: c3b_fstar.json
    python tests/golden/make_golden.py c4       # the warm-start test samples: c4_fstar.json
    python tests/golden/make_golden.py c5       # the radius sweep: c5_fstar.json
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fstar.json")
CONFIGS = {"c0": W.config0, "c1": W.config1, "c2": W.config2}


def main(names):
    gold = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        t = time.time()
        prob = CONFIGS[name]()
        x, res, _ = oracle.reference_solve(prob)
        gold[name] = {
            "workload": prob.name, "n": prob.n, "p": prob.p, "rho": prob.rho,
            "f_star": res.f, "lambda": res.lambda_reg, "l1": res.l1, "fw_gap": res.fw_gap,
            "x_norm2": float(np.linalg.norm(x)), "nnz": int(np.count_nonzero(x)),
            "iters": res.iters, "stop": oracle.STOP_NAMES[res.stop],
        }
        print(name, gold[name], f"{time.time() - t:.1f}s", flush=True)
        with open(OUT, "w") as fh:
            json.dump(gold, fh, indent=1, sort_keys=True)


def main_c3a(count=512):
    """tests/golden/c3a_fstar.json: f* of the ragged batch's instances (the
    oracle's floor solve: iterate until the FP64 line search cannot decrease f)."""
    out = os.path.join(os.path.dirname(OUT), "c3a_fstar.json")
    t = time.time()
    sizes = W.ragged_sizes(count)
    fs = []
    for i, n in enumerate(sizes):
        prob = W.ragged_instance(i, n)
        fs.append(oracle.floor_solve(prob)[1].f)
        if i % 64 == 63:
            print(i + 1, f"{time.time() - t:.0f}s", flush=True)
    with open(out, "w") as fh:
        json.dump({"workload": f"c3a_ragged{count}_bf16", "n": sizes, "f_star": fs,
                   "solver": "oracle.floor_solve"}, fh, indent=0)


def main_c5():
    """tests/golden/c5_fstar.json: f* of each radius of the sweep (workloads.rho_sweep),
    by the oracle's floor solve."""
    out = os.path.join(os.path.dirname(OUT), "c5_fstar.json")
    t = time.time()
    Ks, ldk, n, y, rho, x = W.rho_sweep()
    p = x.shape[0]
    fs = []
    for b, r in enumerate(rho):
        prob = W.Problem(Ks, n, p, ldk, W.DT_BF16, y.copy(), float(r), x, f"c5_{b}")
        fs.append(oracle.floor_solve(prob)[1].f)
        print(b, r, fs[-1], f"{time.time() - t:.0f}s", flush=True)
    with open(out, "w") as fh:
        json.dump({"workload": "c5_rhosweep1848x8192_bf16_50", "rho": [float(r) for r in rho], "f_star": fs,
                   "solver": "oracle.floor_solve"}, fh, indent=0)


def main_c3b(nrhs=1024):
    """tests/golden/c3b_fstar.json: f* of each right-hand side of the shared-K
    workload (K 2048 x 8192 BF16), by the oracle's floor solve."""
    out = os.path.join(os.path.dirname(OUT), "c3b_fstar.json")
    t = time.time()
    Ks, ldk, Y, rho, X = W.shared_k(nrhs=nrhs)
    n, p = Ks.shape[0], X.shape[1]
    fs = []
    for b in range(nrhs):
        prob = W.Problem(Ks, n, p, ldk, W.DT_BF16, Y[b].copy(), float(rho[b]), X[b], f"c3b_{b}")
        fs.append(oracle.floor_solve(prob)[1].f)
        if b % 64 == 63:
            print(b + 1, f"{time.time() - t:.0f}s", flush=True)
    with open(out, "w") as fh:
        json.dump({"workload": f"c3b_sharedK2048x8192_bf16_{nrhs}rhs", "f_star": fs,
                   "solver": "oracle.floor_solve"}, fh, indent=0)


def main_c4():
    """tests/golden/c4_fstar.json: f* of the learned-warm-start workload's test
    samples (the oracle's floor solve of each)."""
    out = os.path.join(os.path.dirname(OUT), "c4_fstar.json")
    t = time.time()
    Ks, ldk, Y, rho, X, ntr = W.warm_start_split()
    n, p = Ks.shape[0], X.shape[1]
    fs = []
    for q in range(ntr, Y.shape[0]):
        prob = W.Problem(Ks, n, p, ldk, W.DT_BF16, Y[q].copy(), float(rho[q]), X[q], f"c4_{q}")
        fs.append(oracle.floor_solve(prob)[1].f)
    print(len(fs), f"{time.time() - t:.0f}s", flush=True)
    with open(out, "w") as fh:
        json.dump({"workload": "c4_warmstart1024x4096_bf16", "first_test_row": ntr, "f_star": fs,
                   "solver": "oracle.floor_solve"}, fh, indent=0)


if __name__ == "__main__":
    args = sys.argv[1:]
    if args == ["c4"]:
        main_c4()
        sys.exit(0)
    if args == ["c5"]:
        main_c5()
        sys.exit(0)
    if args == ["c3a"]:
        main_c3a()
    elif args == ["c3b"]:
        main_c3b()
    else:
        main(args or list(CONFIGS))
