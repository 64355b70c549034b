"""The comparison methods of Sec. 2 (ISTA, FISTA, PSD) on the one-read kernel
against their FP64 oracle (oracle/methods.py), and gpl1_spectral_norm_sq.

  * FP64, config 0: the iterates after 1, 2, 5 and 10 steps equal the
    oracle's to 1e-10 of max|x| (the same arithmetic up to summation order),
    and PSD's last beta/2 equals the oracle's;
  * FP32, config 1: each method stops at the same distance to its optimum as
    Alg. GP + SS in the bench (||K (x - x*)||^2 <= 5e-7 f*: a relative gap of
    5e-7 in f for PSD; for ISTA and FISTA the same absolute gap in eq. 1's
    objective, whose optimum at the stored lambda is f* + 2 lambda rho), and x
    is within 2e-4 of the oracle's x*;
  * the degenerate case lambda >= max|K^T y| (x = 0 is the fixed point) and the
    argument checks of the entry points that run Alg. GP + SS only.
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
from oracle import methods

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
from make_golden import load_sparse  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"
GOLD = os.path.join(os.path.dirname(__file__), "golden")
FSTAR = json.load(open(os.path.join(GOLD, "fstar.json")))
METHODS = [pytest.param(pkg.METHOD_ISTA, id="ista"), pytest.param(pkg.METHOD_FISTA, id="fista"),
           pytest.param(pkg.METHOD_PSD, id="psd")]


def device(prob):
    if prob.dtype == W.DT_BF16:
        return torch.from_numpy(prob.K.view(np.int16)).to(DEV), torch.from_numpy(prob.y).to(DEV)
    return torch.from_numpy(prob.K).to(DEV), torch.from_numpy(prob.y).to(DEV)


def oracle_run(method, K, y, lam, step, rho, iters):
    if method == pkg.METHOD_PSD:
        return methods.psd(K, y, rho, iters)
    return methods.ista(K, y, lam, iters, step=step, fista=method == pkg.METHOD_FISTA)


@pytest.mark.parametrize("method", METHODS)
def test_fp64_iterates_match_the_oracle(gpu_ctx, method):
    prob = W.config0()
    K64 = prob.K_f64()
    lam = FSTAR["c0"]["lambda"]
    step = 1.0 / np.linalg.norm(K64, 2) ** 2
    Kd, yd = device(prob)
    for iters in (1, 2, 5, 10):
        prm = pkg.params_default(stop_rule=0, max_iter=iters, method=method, lambda_pen=lam, step=step)
        x, res = gpu_ctx.solve(Kd, yd, prob.rho, p=prob.p, params=prm)
        torch.cuda.synchronize()
        xo, tr = oracle_run(method, K64, prob.y, lam, step, prob.rho, iters)
        x = x.double().cpu().numpy()
        assert res.iters == iters and res.status == 3, res.as_dict()
        np.testing.assert_allclose(x, xo, rtol=0, atol=1e-10 * np.abs(xo).max())
        if method == pkg.METHOD_PSD:
            assert abs(res.alpha - 0.5 * tr[-1, 2]) <= 1e-9 * tr[-1, 2]
        else:
            assert abs(res.f - methods.penalised(K64, prob.y, lam, x)) <= 1e-9 * res.f


@pytest.mark.parametrize("method", METHODS)
def test_config1_methods_reach_the_optimum(gpu_ctx, method):
    prob = W.config1()
    gold = FSTAR["c1"]
    xs = load_sparse(os.path.join(GOLD, "xstar_c1.npz"))[0][0]
    Kd, yd = device(prob)
    lam, fs = gold["lambda"], gold["f_star"]
    L = gpu_ctx.spectral_norm_sq(Kd, pkg.F32, p=prob.p, iters=100)
    if method == pkg.METHOD_PSD:
        kw = dict(f_star=fs, tol=5e-7)
    else:
        Fs = fs + 2.0 * lam * prob.rho
        kw = dict(f_star=Fs, tol=5e-7 * fs / Fs, lambda_pen=lam, step=1.0 / L)
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, max_iter=20000, method=method, **kw)
    x, res = gpu_ctx.solve(Kd, yd, prob.rho, p=prob.p, params=prm)
    torch.cuda.synchronize()
    x = x.double().cpu().numpy()
    err = np.linalg.norm(x - xs) / np.linalg.norm(xs)
    print(f"method {method}: status {res.status} iters {res.iters} ms {res.kernel_ms:.2f} x err {err:.2e}")
    assert res.status == 0 and res.stop == 0, res.as_dict()
    assert err <= 2e-4 and np.abs(x - xs).max() <= 2e-4 * np.abs(xs).max()


def test_eq1_methods_stop_at_zero_above_lambda_max(gpu_ctx):
    prob = W.config0()
    lam_max = float(np.abs(prob.K_f64().T @ prob.y).max())
    Kd, yd = device(prob)
    for method in (pkg.METHOD_ISTA, pkg.METHOD_FISTA):
        prm = pkg.params_default(stop_rule=0, max_iter=50, method=method, lambda_pen=1.01 * lam_max, step=0.1)
        x, res = gpu_ctx.solve(Kd, yd, prob.rho, p=prob.p, params=prm)
        torch.cuda.synchronize()
        assert res.status == 0 and res.stop == 1 and res.iters == 0, res.as_dict()
        assert torch.count_nonzero(x).item() == 0


def test_methods_are_refused_where_they_do_not_run(gpu_ctx):
    prob = W.config0()
    Kd, yd = device(prob)
    bad = [dict(method=pkg.METHOD_ISTA, lambda_pen=0.1, step=0.1, engine=pkg.ENGINE_TWO_PASS),
           dict(method=pkg.METHOD_ISTA, lambda_pen=0.0, step=0.1),
           dict(method=pkg.METHOD_FISTA, lambda_pen=0.1, step=-1.0),
           dict(method=pkg.METHOD_ISTA, lambda_pen=0.1, step=0.1, stop_rule=pkg.STOP_ON_FW),
           dict(method=7)]
    for kw in bad:
        with pytest.raises(pkg.Gpl1Error):
            gpu_ctx.solve(Kd, yd, prob.rho, p=prob.p, params=pkg.params_default(**kw))
    x = torch.zeros(prob.p, dtype=torch.float64, device=DEV)
    desc = [pkg.Context.make_problem(Kd, yd, prob.rho, x, prob.p)]
    with pytest.raises(pkg.Gpl1Error):
        gpu_ctx.solve_batched(desc, W.DT_F64, pkg.params_default(method=pkg.METHOD_PSD))


@pytest.mark.parametrize("dtype,n,p", [(W.DT_F64, 256, 1024), (W.DT_F32, 512, 2048), (W.DT_BF16, 1024, 4096)])
def test_spectral_norm_sq_against_the_svd(gpu_ctx, dtype, n, p):
    """The estimate lies below ||K||_2^2 (a Rayleigh quotient) and within 1e-3 of it."""
    prob = W.gaussian(n, p, 10, dtype=dtype, seed=3 + n)
    exact = np.linalg.norm(prob.K_f64(), 2) ** 2
    Kd, _ = device(prob)
    est = gpu_ctx.spectral_norm_sq(Kd, dtype, p=p, iters=200)
    print(f"{dtype} {n}x{p}: {est:.9g} vs {exact:.9g}")
    assert est <= exact * (1 + 1e-6) and est >= exact * (1 - 1e-3)
