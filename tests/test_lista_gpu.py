"""Learned warm start (gpl1_lista_*): forward and gradients against the FP64
oracle (oracle/lista.py) on the same K and weights, training lowering the loss,
and the trained network's projected output cutting Alg. GP's iterations.

Tolerances: the products run with BF16 operands (unit roundoff 2^-9) over a
few layers, so x^L and the gradients carry relative errors of a few 1e-3 per
rounding and up to ~1e-2 after the layers compound; the bars below are 4e-2
for x^L and the loss and 1e-1 for the gradients (with cosine >= 0.99)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import lista as OL
import paper_0902_4424_gb300 as pkg
import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def setup(n, p, B, L, seed):
    Ks, ldk, Y, rho, X = W.warm_start_data(n, p, B, max(2, n // 20), seed=seed)
    K64 = W.bf16_bits_to_f64(Ks[:, :p])
    rng = np.random.default_rng(seed)
    W0, th0, Lk = OL.init_params(K64, L, 0.05)
    Wp = (W0 * (1 + 0.2 * rng.standard_normal(W0.shape))).astype(np.float32)
    th = (th0 * (1 + 0.3 * rng.random(L))).astype(np.float32)
    dev = dict(K=torch.from_numpy(Ks.view(np.int16)).to(DEV), W=torch.from_numpy(Wp).to(DEV),
               th=torch.from_numpy(th).to(DEV), Y=torch.from_numpy(Y).to(DEV),
               Xt=torch.from_numpy(X.astype(np.float32)).to(DEV))
    return K64, Wp.astype(np.float64), th.astype(np.float64), Y.astype(np.float64), X, dev


def test_lista_forward_matches_oracle(gpu_ctx):
    K64, Wp, th, Y, X, d = setup(128, 512, 64, 4, 71)
    xg = gpu_ctx.lista_forward(d["K"], d["W"], d["th"], d["Y"]).double().cpu().numpy()
    xo = OL.forward(K64, Wp, th, Y)[0][-1]
    assert np.linalg.norm(xg - xo) <= 4e-2 * np.linalg.norm(xo)


def test_lista_gradients_match_oracle(gpu_ctx):
    K64, Wp, th, Y, X, d = setup(128, 512, 64, 3, 72)
    loss, dW, dth = gpu_ctx.lista_grad(d["K"], d["W"], d["th"], d["Y"], d["Xt"])
    lo, dWo, dtho = OL.backward(K64, Wp, th, Y, X)
    assert abs(loss - lo) <= 4e-2 * lo
    g, o = dW.double().cpu().numpy().ravel(), dWo.ravel()
    assert np.linalg.norm(g - o) <= 1e-1 * np.linalg.norm(o)
    assert g @ o >= 0.99 * np.linalg.norm(g) * np.linalg.norm(o)
    t = dth.double().cpu().numpy()
    assert np.all(np.abs(t - dtho) <= 1e-1 * np.abs(dtho).max())


def test_lista_training_lowers_the_loss(gpu_ctx):
    n, p, N, L = 128, 512, 1024, 4
    K64, Wp, th, Y, X, d = setup(n, p, N, L, 73)
    m = torch.zeros(L * p * n + L, dtype=torch.float32, device=DEV)
    v = torch.zeros_like(m)
    losses = gpu_ctx.lista_train(d["K"], d["W"], d["th"], m, v, d["Y"], d["Xt"], batch=64, steps=160,
                                 lr=2e-4, lr_theta=1e-4)
    assert all(np.isfinite(losses))
    assert np.mean(losses[-16:]) < 0.75 * np.mean(losses[:16]), (losses[:4], losses[-4:])


def test_lista_warm_start_cuts_gp_iterations(gpu_ctx):
    """Train on solutions of eq. 2 from the solver itself, then start Alg. GP from
    the projected network output: fewer iterations to the same 5e-7 gap."""
    n, p, L, k = 256, 1024, 6, 12
    Ntr, Nte = 2048, 12
    Ks, ldk, Y, rho, Xtrue = W.warm_start_data(n, p, Ntr + Nte, k, seed=74)
    K = torch.from_numpy(Ks.view(np.int16)).to(DEV)
    Yd = torch.from_numpy(Y).to(DEV)
    # training targets: the solver's solutions (shared-K form, run to its floor)
    Xs, res = gpu_ctx.solve_shared_k(K, Yd[:Ntr], rho[:Ntr], p=p,
                                     params=pkg.params_default(stop_rule=0, max_iter=150))
    K64 = W.bf16_bits_to_f64(Ks[:, :p])
    W0, th0, Lk = OL.init_params(K64, L, 0.02)
    Wd = torch.from_numpy(W0.astype(np.float32)).to(DEV)
    thd = torch.from_numpy(th0.astype(np.float32)).to(DEV)
    m = torch.zeros(L * p * n + L, dtype=torch.float32, device=DEV)
    v = torch.zeros_like(m)
    losses = gpu_ctx.lista_train(K, Wd, thd, m, v, Yd[:Ntr], Xs, batch=256, steps=400, lr=1e-4, lr_theta=1e-4)
    assert np.mean(losses[-8:]) < np.mean(losses[:8])
    pad = torch.zeros(64, n, dtype=torch.float32, device=DEV)          # the batch must be a multiple of 64
    pad[:Nte] = Yd[Ntr:]
    x0 = gpu_ctx.lista_forward(K, Wd, thd, pad)[:Nte]
    cold, warm = [], []
    for q in range(Nte):
        b = Ntr + q
        prob = W.Problem(Ks, n, p, ldk, W.DT_BF16, Y[b].copy(), float(rho[b]), Xtrue[b], f"w{q}")
        fs = oracle.reference_solve(prob)[1].f
        prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, f_star=fs, max_iter=5000)
        _, rc = gpu_ctx.solve(K, Yd[b], float(rho[b]), p=p, params=prm)
        xw, rw = gpu_ctx.solve(K, Yd[b], float(rho[b]), x=x0[q].clone(), p=p, params=prm)
        torch.cuda.synchronize()
        assert rc.status == 0 and rw.status == 0, (rc.as_dict(), rw.as_dict())
        assert (oracle.objective(prob, xw.double().cpu().numpy()) - fs) / fs <= 1e-6
        cold.append(rc.iters)
        warm.append(rw.iters)
    assert np.mean(warm) < np.mean(cold), (cold, warm)
