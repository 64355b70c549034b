"""The learned warm start as a product (gpl1_lista_init, gpl1_solve_warm):

  * the initial network is one ISTA step of eq. 1 per layer: W_l = K^T (1/L)
    entry by entry in FP32 (K widened exactly from BF16), theta_l =
    median(lambdas) / L, with L within 1e-3 of ||K||_2^2 from the SVD;
  * warm solves from that network reach the oracle's optima (relative gap
    <= 1e-6 in FP64) with no fallback, for a batch whose size is not a multiple
    of 64 (the ragged tail of the network pass);
  * a deliberately poor network (large random weights) with a two-iteration
    warm budget leaves the warm solves unconverged: every one falls back to the
    cold solve, which still reaches the oracle's optimum.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_0902_4424_gb300 as pkg
import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def case(n=256, p=1024, nrhs=200, k=12, seed=91):
    """Instances drawn like the shared-K tests' (+-1 signals, noise 0.01)."""
    Ks, ldk, Y, rho, X = W.shared_k(n, p, nrhs, k, seed=seed)
    probs = [W.Problem(Ks, n, p, ldk, W.DT_BF16, Y[b].copy(), float(rho[b]), X[b], f"w{b}") for b in range(nrhs)]
    return Ks, ldk, Y, rho, probs


def test_lista_init_is_one_ista_step_per_layer(gpu_ctx):
    Ks, ldk, Y, rho, probs = case(nrhs=1)
    n, p = Ks.shape[0], probs[0].p
    K = torch.from_numpy(Ks.view(np.int16)).to(DEV)
    lams = [0.3, 0.1, 0.2, 0.7]
    Wd, th, L = gpu_ctx.lista_init(K, 3, lams, p=p)
    K64 = W.bf16_bits_to_f64(Ks[:, :p])
    exact = np.linalg.norm(K64, 2) ** 2
    assert exact * (1 - 1e-3) <= L <= exact * (1 + 1e-6)
    Wh = Wd.double().cpu().numpy()
    for l in range(3):
        np.testing.assert_array_equal(Wh[l], K64.T.astype(np.float32) * np.float32(1.0 / L))
    np.testing.assert_array_equal(th.cpu().numpy(), np.full(3, np.float32(0.25 / L)))


def solve_all(ctx, Ks, Y, rho, probs, Wd, th, fstars, warm_max_iter):
    K = torch.from_numpy(Ks.view(np.int16)).to(DEV)
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).to(DEV)
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, max_iter=5000)
    X, res, fb, nfb = ctx.solve_warm(K, Wd, th, Yd, rho, f_star=fstars, params=prm, warm_max_iter=warm_max_iter)
    torch.cuda.synchronize()
    Xh = X.double().cpu().numpy()
    for pr, x, r, fs in zip(probs, Xh, res, fstars):
        assert r.status == 0, r.as_dict()
        assert (oracle.objective(pr, x) - fs) / fs <= 1e-6
        assert np.abs(x).sum() <= pr.rho * (1 + 1e-6)
    return res, fb, nfb


def test_warm_solves_reach_the_optima_without_fallback(gpu_ctx):
    Ks, ldk, Y, rho, probs = case()
    fstars = [oracle.reference_solve(pr)[1].f for pr in probs]
    K = torch.from_numpy(Ks.view(np.int16)).to(DEV)
    Wd, th, L = gpu_ctx.lista_init(K, 4, [0.02], p=probs[0].p)
    res, fb, nfb = solve_all(gpu_ctx, Ks, Y, rho, probs, Wd, th, fstars, warm_max_iter=0)
    assert nfb == 0 and not any(fb)


def test_poor_network_falls_back_to_the_cold_solve(gpu_ctx):
    Ks, ldk, Y, rho, probs = case(nrhs=70)
    fstars = [oracle.reference_solve(pr)[1].f for pr in probs]
    n, p = Ks.shape[0], probs[0].p
    g = torch.Generator().manual_seed(5)
    Wd = (10.0 * torch.randn(3, p, n, generator=g)).to(DEV)
    th = torch.zeros(3, dtype=torch.float32, device=DEV)
    res, fb, nfb = solve_all(gpu_ctx, Ks, Y, rho, probs, Wd, th, fstars, warm_max_iter=2)
    assert nfb == len(probs) and all(fb)
