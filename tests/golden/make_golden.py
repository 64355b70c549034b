"""Write tests/golden/fstar.json: optimal objective values of the measured configurations.

Every number here comes from the FP64 oracle (oracle/) run on the seeded
inputs of workloads/ to its precision floor (Frank-Wolfe certificate 1e-13 or
no decrease of f for 30 iterations).  Nothing here touches the CUDA path.

    python tests/golden/make_golden.py [c0 c1 c2 ...]
    python tests/golden/make_golden.py c3a      # the ragged batch: c3a_fstar.json
    python tests/golden/make_golden.py c3b      # the shared-K right-hand sides: c3b_fstar.json
    python tests/golden/make_golden.py c4       # the warm-start test samples: c4_fstar.json
    python tests/golden/make_golden.py c5       # the radius sweep: c5_fstar.json
    python tests/golden/make_golden.py xstar    # the oracle's solutions x*: xstar_*.npz
    python tests/golden/make_golden.py homotopy # exact minimisers from the homotopy path
    python tests/golden/make_golden.py c4full   # f* of the 10^4 warm-start test samples

The x* files hold each solution sparsely (indices and values of its nonzero
entries, FP64), for configs 0-2 and for a seeded sample of the instances of
the ragged batch, the shared-K right-hand sides, the warm-start test samples
and the radius sweep.  Each comes from the same oracle run as the stored f*
(the reference solve for configs 0-2, the floor solve for the rest), so
f(x*) equals the stored f*.

The homotopy files hold exact minimisers from the oracle's homotopy path
(oracle/homotopy.py, no iteration): homotopy_small.npz for six small FP64
problems (workloads.homotopy_case; y stored with them, so that no platform's
matrix product enters), and xbar_c5.npz for every radius of the radius sweep.
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
WORKLOAD_OF = {"c0": W.config0, "c1": W.config1, "c2": W.config2}


def main(names):
    gold = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        t = time.time()
        prob = WORKLOAD_OF[name]()
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


def _save_sparse(path, xs, meta):
    """xs: list of FP64 vectors; stored as their nonzero entries."""
    arrs = {}
    for i, x in enumerate(xs):
        nz = np.flatnonzero(x)
        arrs[f"idx{i}"] = nz.astype(np.int32)
        arrs[f"val{i}"] = x[nz]
        arrs[f"p{i}"] = np.array([x.shape[0]])
    np.savez_compressed(path, count=np.array([len(xs)]), meta=np.array(json.dumps(meta)), **arrs)


def load_sparse(path):
    """(list of dense FP64 vectors, meta dict) from a file written by _save_sparse."""
    z = np.load(path)
    xs = []
    for i in range(int(z["count"][0])):
        x = np.zeros(int(z[f"p{i}"][0]))
        x[z[f"idx{i}"]] = z[f"val{i}"]
        xs.append(x)
    return xs, json.loads(str(z["meta"]))


SAMPLE = 16   # instances per sampled workload


def main_xstar(which=("c0", "c1", "c2", "c3a", "c3b", "c4", "c5")):
    """tests/golden/xstar_<cfg>.npz: the oracle's x* (same solves as the f* files)."""
    d = os.path.dirname(OUT)
    gold = json.load(open(OUT))
    for name in which:
        t = time.time()
        if name in WORKLOAD_OF:
            prob = WORKLOAD_OF[name]()
            x, res, _ = oracle.reference_solve(prob)
            meta = {"workload": prob.name, "f": res.f, "f_star_file": gold[name]["f_star"], "solver": "oracle.reference_solve"}
            _save_sparse(os.path.join(d, f"xstar_{name}.npz"), [x], meta)
        elif name == "c3a":
            sizes = W.ragged_sizes(512)
            idx = list(range(0, 512, 512 // SAMPLE))
            xs, fs = [], []
            for i in idx:
                x, r, _ = oracle.floor_solve(W.ragged_instance(i, sizes[i]))
                xs.append(x)
                fs.append(r.f)
            _save_sparse(os.path.join(d, "xstar_c3a.npz"), xs, {"instances": idx, "f": fs, "solver": "oracle.floor_solve"})
        elif name == "c3b":
            Ks, ldk, Y, rho, X = W.shared_k(nrhs=1024)
            n, p = Ks.shape[0], X.shape[1]
            idx = list(range(0, 1024, 1024 // SAMPLE))
            xs, fs = [], []
            for b in idx:
                x, r, _ = oracle.floor_solve(W.Problem(Ks, n, p, ldk, W.DT_BF16, Y[b].copy(), float(rho[b]), X[b], "c3b"))
                xs.append(x)
                fs.append(r.f)
            _save_sparse(os.path.join(d, "xstar_c3b.npz"), xs, {"instances": idx, "f": fs, "solver": "oracle.floor_solve"})
        elif name == "c4":
            Ks, ldk, Y, rho, X, ntr = W.warm_start_split()
            n, p = Ks.shape[0], X.shape[1]
            nte = Y.shape[0] - ntr
            idx = list(range(0, nte, nte // SAMPLE))
            xs, fs = [], []
            for q in idx:
                x, r, _ = oracle.floor_solve(W.Problem(Ks, n, p, ldk, W.DT_BF16, Y[ntr + q].copy(), float(rho[ntr + q]),
                                                       X[ntr + q], "c4"))
                xs.append(x)
                fs.append(r.f)
            _save_sparse(os.path.join(d, "xstar_c4.npz"), xs, {"test_samples": idx, "f": fs, "solver": "oracle.floor_solve"})
        elif name == "c5":
            Ks, ldk, n, y, rho, xt = W.rho_sweep()
            p = xt.shape[0]
            idx = list(range(0, len(rho), 5))
            xs, fs = [], []
            for b in idx:
                x, r, _ = oracle.floor_solve(W.Problem(Ks, n, p, ldk, W.DT_BF16, y.copy(), float(rho[b]), xt, "c5"))
                xs.append(x)
                fs.append(r.f)
            _save_sparse(os.path.join(d, "xstar_c5.npz"), xs, {"radii": idx, "f": fs, "solver": "oracle.floor_solve"})
        print(name, f"{time.time() - t:.0f}s", flush=True)


_C4 = {}


def _c4full_init():
    oracle.set_threads(1)
    _C4["K"], _C4["ldk"] = W.warm_start_K()
    _C4["Y"], _C4["rho"] = W.warm_start_test()


def _c4full_one(q):
    Ks, ldk = _C4["K"], _C4["ldk"]
    prob = W.Problem(Ks, Ks.shape[0], 4096, ldk, W.DT_BF16, _C4["Y"][q].copy(), float(_C4["rho"][q]), None, "c4f")
    return oracle.floor_solve(prob)[1].f


def main_c4full(procs=8):
    """tests/golden/c4full_fstar.json: f* of the 10^4 test samples of the full
    learned-warm-start configuration (workloads.warm_start_test), by the oracle's
    floor solve, one single-threaded solve per worker process."""
    import multiprocessing as mp
    out = os.path.join(os.path.dirname(OUT), "c4full_fstar.json")
    t = time.time()
    count = W.WARM_TEST_FULL
    with mp.get_context("spawn").Pool(procs, initializer=_c4full_init) as pool:
        fs = pool.map(_c4full_one, range(count), chunksize=16)
    print(len(fs), f"{time.time() - t:.0f}s", flush=True)
    with open(out, "w") as fh:
        json.dump({"workload": f"c4_warmstart1024x4096_bf16_test{count}", "f_star": fs,
                   "solver": "oracle.floor_solve"}, fh, indent=0)


HOMOTOPY_CASES = [(0, 30, 60, 6), (1, 30, 60, 6), (2, 40, 120, 8), (3, 50, 40, 5), (4, 20, 200, 4),
                  (5, 64, 64, 10)]


def main_homotopy():
    """tests/golden/homotopy_small.npz and tests/golden/xbar_c5.npz (exact path points)."""
    from oracle import homotopy
    d = os.path.dirname(OUT)
    t = time.time()
    arrs = {}
    for q, (seed, n, p, k) in enumerate(HOMOTOPY_CASES):
        K, y, rho, _ = W.homotopy_case(seed, n, p, k)
        xh, lam, segs = homotopy.solve_at_radius(K, y, rho)
        arrs.update({f"y{q}": y, f"x{q}": xh, f"lam{q}": np.array([lam]), f"rho{q}": np.array([rho])})
    np.savez_compressed(os.path.join(d, "homotopy_small.npz"), cases=np.array(HOMOTOPY_CASES), **arrs)
    Ks, ldk, n, y, rho, xt = W.rho_sweep()
    p = xt.shape[0]
    sols = homotopy.solve_at_radii(W.bf16_bits_to_f64(Ks[:, :p]), y.astype(np.float64), rho)
    _save_sparse(os.path.join(d, "xbar_c5.npz"), [s[0] for s in sols],
                 {"radii": list(range(len(rho))), "lam": [s[1] for s in sols], "segments": [s[2] for s in sols],
                  "solver": "oracle.homotopy.solve_at_radii"})
    print("homotopy", f"{time.time() - t:.0f}s", flush=True)


if __name__ == "__main__":
    args = sys.argv[1:]
    if args == ["c4full"]:
        main_c4full()
        sys.exit(0)
    if args == ["homotopy"]:
        main_homotopy()
        sys.exit(0)
    if args and args[0] == "xstar":
        main_xstar(tuple(args[1:]) or ("c0", "c1", "c2", "c3a", "c3b", "c4", "c5"))
        sys.exit(0)
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
        main(args or list(WORKLOAD_OF))
