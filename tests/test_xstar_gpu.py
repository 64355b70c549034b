"""The returned x against the oracle's minimiser x* at the measured sizes.

A relative objective gap of 1e-6 bounds ||K (x - x*)||, not ||x - x*||, so a
wrong support could pass a gap test; these compare x itself with the oracle's
x* (tests/golden/xstar_*.npz, written by make_golden.py from oracle/ alone) and
with the exact minimisers of the homotopy path (homotopy_small.npz,
xbar_c5.npz).  Bars, as the method is specified for these workloads:

  * ||x - x*|| / ||x*|| <= 1e-4;
  * max_i |x_i - x*_i| <= 1e-4 max|x*| (no entry carries the error alone);
  * support and sign: every entry with |x*_i| > 1e-3 max|x*| has the sign of
    x*_i in x, and no entry where x*_i = 0 exceeds 1e-3 max|x*| in x (the
    lambda-rho relation of Sec. 1 fixes the signs on the support).

x* is unique on every workload here (K in general position; for config 2, K is
square and of full rank), and each kernel stops at the bench's 5e-7 relative
gap except where a gap in f says little about x:
  * config 2: K has singular values down to 1e-4; it is solved at a tightened
    stop (relative gap 1e-8) before x is compared;
  * the radius sweep: at the small radii f* is most of ||y||^2 while ||K x*||
    is small, so ||K (x - x*)||^2 <= gap f* leaves x loose; every radius runs a
    fixed 500 iterations (no gap stop) before x is compared.
"""
import json
import os
import sys

import numpy as np
import pytest
import torch

import oracle
import paper_0902_4424_gb300 as pkg
import workloads as W

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
from make_golden import HOMOTOPY_CASES, load_sparse  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"
GOLD = os.path.join(os.path.dirname(__file__), "golden")
FSTAR = json.load(open(os.path.join(GOLD, "fstar.json")))
ENGINES = [pytest.param(pkg.ENGINE_ONE_READ, id="one_read"), pytest.param(pkg.ENGINE_TWO_PASS, id="two_pass")]


def fstars(name):
    return json.load(open(os.path.join(GOLD, f"{name}_fstar.json")))["f_star"]


def x_errors(x, xs):
    """(relative 2-norm error, max entry error / max|x*|, sign mismatches on the
    support of x*, entries of x above the support threshold where x* is zero)."""
    x = np.asarray(x, np.float64)
    m = np.abs(xs).max()
    big = np.abs(xs) > 1e-3 * m
    rel = np.linalg.norm(x - xs) / np.linalg.norm(xs)
    emax = np.abs(x - xs).max() / m
    bad_sign = int(np.sum(np.sign(x[big]) != np.sign(xs[big])))
    extra = int(np.sum((np.abs(x) > 1e-3 * m) & (xs == 0)))
    return rel, emax, bad_sign, extra


def assert_x_close(x, xs, what, rel_bar=1e-4, max_bar=1e-4):
    rel, emax, bad_sign, extra = x_errors(x, xs)
    print(f"{what}: rel {rel:.2e} max {emax:.2e} sign {bad_sign} extra {extra}")
    assert rel <= rel_bar and emax <= max_bar and bad_sign == 0 and extra == 0, (what, rel, emax, bad_sign, extra)


def device_K(prob):
    if prob.dtype == W.DT_BF16:
        return torch.from_numpy(prob.K.view(np.int16)).to(DEV)
    return torch.from_numpy(prob.K).to(DEV)


@pytest.mark.parametrize("engine", ENGINES)
def test_config1_x_matches_oracle(gpu_ctx, engine):
    """K 4096 x 16384 FP32, stopped at the bench's 5e-7 gap."""
    prob = W.config1()
    xs = load_sparse(os.path.join(GOLD, "xstar_c1.npz"))[0][0]
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, f_star=FSTAR["c1"]["f_star"],
                             max_iter=20000, engine=engine)
    x, res = gpu_ctx.solve(device_K(prob), torch.from_numpy(prob.y).to(DEV), prob.rho, p=prob.p, params=prm)
    torch.cuda.synchronize()
    assert res.status == 0, res.as_dict()
    assert_x_close(x.double().cpu().numpy(), xs, "c1")


@pytest.mark.parametrize("engine", ENGINES)
def test_config2_x_matches_oracle_at_tightened_stop(gpu_ctx, engine):
    """K 4096 x 4096 FP32 with singular values from 1 to 1e-4: x compared after
    the tightened stop (relative gap 1e-8), and the Sec. 1 conditions on the
    support at a bar of 5e-3 of lambda.  On the support the correlation at x*
    equals lambda* sgn x*, so the residual at x is the difference of the two
    correlations, (K^T K (x - x*))_i, over lambda (plus x*'s own residual and
    lambda - lambda*): with x within the 1e-4 bar of x* that reaches a few
    1e-3 of lambda on this operator (measured 0.6e-3 to 1.6e-3)."""
    prob = W.config2()
    xs = load_sparse(os.path.join(GOLD, "xstar_c2.npz"))[0][0]
    fs = FSTAR["c2"]["f_star"]
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=1e-8, f_star=fs, max_iter=20000, engine=engine)
    x, res = gpu_ctx.solve(device_K(prob), torch.from_numpy(prob.y).to(DEV), prob.rho, p=prob.p, params=prm)
    torch.cuda.synchronize()
    xh = x.double().cpu().numpy()
    gap = (oracle.objective(prob, xh) - fs) / fs
    print(f"c2: status {res.status} iters {res.iters} gap {gap:.2e}")
    # at 1e-8 the FP32 kernel's own f may not resolve the gap: it ends at the
    # rule or, at its precision floor, by the stagnation stop; x is what counts
    assert res.status == 0 or (res.status == 3 and res.stop == 5), res.as_dict()
    assert_x_close(xh, xs, "c2")
    f, lam, fw, g = oracle.certificates(prob, xh)
    c = -0.5 * g
    supp = np.abs(xs) > 1e-3 * np.abs(xs).max()
    kkt = np.abs(c[supp] - lam * np.sign(xh[supp])).max() / lam
    _, lam_s, _, g_s = oracle.certificates(prob, xs)
    dc = 0.5 * np.abs(g[supp] - g_s[supp]).max() / lam   # |(K^T K (x - x*))_i| / lambda
    print(f"c2: KKT {kkt:.2e} (correlation difference {dc:.2e}, lambda {lam:.4e} vs {lam_s:.4e})")
    assert kkt <= 5e-3


def test_ragged_batch_sample_x_matches_oracle(gpu_ctx):
    """Every 32nd instance of the 512-instance ragged batch (n 128..2048, p = 4n,
    BF16), solved together in one gpl1_solve_batched call."""
    xsl, meta = load_sparse(os.path.join(GOLD, "xstar_c3a.npz"))
    sizes = W.ragged_sizes(512)
    fs = fstars("c3a")
    keep, descs, probs = [], [], []
    for i in meta["instances"]:
        pr = W.ragged_instance(i, sizes[i])
        K, y = device_K(pr), torch.from_numpy(pr.y).to(DEV)
        x = torch.zeros(pr.p, dtype=torch.float32, device=DEV)
        keep.append((K, y, x))
        probs.append(pr)
        descs.append(pkg.Context.make_problem(K, y, pr.rho, x, pr.p, fs[i]))
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, x0_is_zero=1, max_iter=20000)
    res = gpu_ctx.solve_batched(descs, W.DT_BF16, prm)
    torch.cuda.synchronize()
    for i, pr, (_, _, x), xs, r in zip(meta["instances"], probs, keep, xsl, res):
        assert r.status == 0, (i, r.as_dict())
        assert_x_close(x.double().cpu().numpy(), xs, f"c3a[{i}] n={pr.n}")


def test_shared_k_sample_x_matches_oracle(gpu_ctx):
    """The shared-K workload at full size (1024 right-hand sides on one BF16 K
    2048 x 8192, tensor-core products): every 64th right-hand side's x."""
    xsl, meta = load_sparse(os.path.join(GOLD, "xstar_c3b.npz"))
    fs = fstars("c3b")
    Ks, ldk, Y, rho, Xt = W.shared_k(nrhs=len(fs))
    K = torch.from_numpy(Ks.view(np.int16)).to(DEV)
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).to(DEV)
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, max_iter=2000)
    X, res = gpu_ctx.solve_shared_k(K, Yd, rho, p=Xt.shape[1], f_star=fs, params=prm)
    torch.cuda.synchronize()
    Xh = X.double().cpu().numpy()
    for b, xs in zip(meta["instances"], xsl):
        assert res[b].status == 0, (b, res[b].as_dict())
        assert_x_close(Xh[b], xs, f"c3b[{b}]")


def test_warm_start_test_sample_x_matches_oracle(gpu_ctx):
    """Every 16th test sample of the learned-warm-start workload (K 1024 x 4096
    BF16, 50-sparse Gaussian signals), each by gpl1_solve."""
    xsl, meta = load_sparse(os.path.join(GOLD, "xstar_c4.npz"))
    fs = fstars("c4")
    Ks, ldk, Y, rho, Xt, ntr = W.warm_start_split()
    K = torch.from_numpy(Ks.view(np.int16)).to(DEV)
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).to(DEV)
    for q, xs in zip(meta["test_samples"], xsl):
        prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, f_star=fs[q], max_iter=20000)
        x, r = gpu_ctx.solve(K, Yd[ntr + q], float(rho[ntr + q]), p=Xt.shape[1], params=prm)
        torch.cuda.synchronize()
        assert r.status == 0, (q, r.as_dict())
        assert_x_close(x.double().cpu().numpy(), xs, f"c4[{q}]")


def test_radius_sweep_x_matches_oracle_and_homotopy(gpu_ctx):
    """All 50 radii of the sweep in one shared-K call of 500 iterations each:
    every 5th radius against the oracle's Alg. GP solution, and every radius
    against the exact point of the homotopy path (x-bar of the isochrones of
    Sec. 4)."""
    xsl, meta = load_sparse(os.path.join(GOLD, "xstar_c5.npz"))
    xbar, hmeta = load_sparse(os.path.join(GOLD, "xbar_c5.npz"))
    fs = fstars("c5")
    Ks, ldk, n, y, rho, xt = W.rho_sweep()
    R = len(rho)
    K = torch.from_numpy(Ks.view(np.int16)).to(DEV)
    Yd = torch.from_numpy(y).to(DEV).unsqueeze(0).repeat(R, 1).contiguous()
    prm = pkg.params_default(stop_rule=0, max_iter=500)
    X, res = gpu_ctx.solve_shared_k(K, Yd, rho, p=xt.shape[0], params=prm)
    torch.cuda.synchronize()
    Xh = X.double().cpu().numpy()
    for r in res:
        assert r.stop in (1, 3) and r.status in (0, 3), r.as_dict()   # stationary, or max_iter
    for b, xs in zip(meta["radii"], xsl):
        assert_x_close(Xh[b], xs, f"c5[{b}] vs Alg. GP")
    for b in range(R):
        assert_x_close(Xh[b], xbar[b], f"c5[{b}] vs homotopy")


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("case", range(len(HOMOTOPY_CASES)))
def test_fp64_solve_matches_the_exact_homotopy_path(gpu_ctx, case, engine):
    """The FP64 path against the exact minimiser from the homotopy path (no
    iteration on the reference side; stored with its y by make_golden.py): the
    same support and signs, x to 1e-6, f to 1e-9."""
    seed, n, p, k = HOMOTOPY_CASES[case]
    K, _, _, xt = W.homotopy_case(seed, n, p, k)
    z = np.load(os.path.join(GOLD, "homotopy_small.npz"))
    y, xh, rho = z[f"y{case}"], z[f"x{case}"], float(z[f"rho{case}"][0])
    fh = float(np.sum((K @ xh - y) ** 2))
    prob = W.Problem(np.ascontiguousarray(K), n, p, p, W.DT_F64, y, rho, xt, "homotopy")
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=1e-12, f_star=fh, max_iter=100000, engine=engine)
    x, res = gpu_ctx.solve(torch.from_numpy(prob.K).to(DEV), torch.from_numpy(y).to(DEV), rho, p=p, params=prm)
    torch.cuda.synchronize()
    x = x.double().cpu().numpy()
    assert res.status == 0, res.as_dict()
    assert abs(oracle.objective(prob, x) - fh) <= 1e-9 * fh
    assert np.linalg.norm(x - xh) <= 1e-6 * np.linalg.norm(xh)
    assert np.array_equal(np.sign(xh), np.sign(np.where(np.abs(x) > 1e-9 * np.abs(x).max(), x, 0.0)))
