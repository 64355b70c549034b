"""Learned warm start (gpl1_lista_*): forward and gradients against the FP64
oracle (oracle/lista.py) on the same K and weights, training lowering the loss,
and the trained network's projected output cutting Alg. GP's iterations.

Two comparisons.  Element by element against the oracle's BF16 precision
model (the same operands rounded to BF16 as the kernels round them, the same
FP32 elementwise steps): the kernels differ from it only by the order of their
FP32 accumulations, which moves a value by ~1e-7 relative and, rarely, flips
a BF16 rounding or a threshold mask (one 2^-8 step of one entry, carried into
the later layers); the bars are on the 99.9th percentile of the per-entry
error, its maximum and the per-layer Frobenius error.  On data that no
rounding touches the kernels must agree exactly.  And, as the
accuracy statement, against the unrounded FP64 network: BF16 operands (unit
roundoff 2^-9) over a few layers give relative errors of a few 1e-3 per
rounding and ~1e-2 after the layers compound; the bars there are 4e-2 for
x^L and the loss and 1e-1 for the gradients (with cosine >= 0.99)."""
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


def entrywise(g, e):
    """(99.9th percentile, maximum) of |g - e| over the entries, relative to max |e|."""
    err = np.abs(np.asarray(g, np.float64) - e).ravel()
    scale = np.abs(e).max()
    return float(np.quantile(err, 0.999) / scale), float(err.max() / scale)


def test_lista_exact_on_representable_data(gpu_ctx):
    """On data whose every operand is a short dyadic fraction (workloads.
    lista_exact_case: BF16 operands and FP32 sums lose nothing, which the
    oracle's pins confirm), the kernels must return the FP64 network's x^L, loss,
    dW and dtheta exactly: any dropped or mis-signed term, wrong index or
    transposed operand shows here as an exact mismatch."""
    K, Wt, th, Y, Xt = W.lista_exact_case()
    L = Wt.shape[0]
    Kd = torch.from_numpy(K.astype(np.float32)).to(torch.bfloat16).view(torch.int16).to(DEV)
    Wd = torch.from_numpy(Wt.astype(np.float32)).to(DEV)
    thd = torch.from_numpy(th.astype(np.float32)).to(DEV)
    Yd = torch.from_numpy(Y.astype(np.float32)).to(DEV)
    Xd = torch.from_numpy(Xt.astype(np.float32)).to(DEV)
    xs, _ = OL.forward(K, Wt, th, Y)
    xg = gpu_ctx.lista_forward(Kd, Wd, thd, Yd).double().cpu().numpy()
    assert np.array_equal(xg, xs[-1]), np.abs(xg - xs[-1]).max()
    lo, dWo, dtho = OL.backward(K, Wt, th, Y, Xt)
    loss, dW, dth = gpu_ctx.lista_grad(Kd, Wd, thd, Yd, Xd)
    assert loss == lo, (loss, lo)
    for l in range(L):
        g = dW[l].double().cpu().numpy()
        assert np.array_equal(g, dWo[l]), (l, int(np.sum(g != dWo[l])), np.abs(g - dWo[l]).max())
    assert np.array_equal(dth.double().cpu().numpy(), dtho), (dth, dtho)


@pytest.mark.parametrize("n,p,B,L", [(128, 512, 64, 4), (1024, 4096, 64, 6)])
def test_lista_matches_bf16_precision_model_entrywise(gpu_ctx, n, p, B, L):
    """Forward output and both gradients entry by entry against the oracle's
    BF16 precision model, at a small shape and at the warm-start workload's
    shape (K 1024 x 4096, 6 layers).  A threshold mask that flips between the
    two (|z| within the FP32 noise of theta) moves one delta entry by a whole
    gradient value, so the maximum error of dW is bounded loosely and the bulk
    tightly: the 99.9th percentile per entry, and the Frobenius error of every
    layer separately (a wrong layer would show there)."""
    K64, Wp, th, Y, X, d = setup(n, p, B, L, 75 + n)
    xg = gpu_ctx.lista_forward(d["K"], d["W"], d["th"], d["Y"]).double().cpu().numpy()
    xe = OL.forward(K64, Wp, th, Y, rounded=True)[0][-1]
    q, m = entrywise(xg, xe)
    print(f"x^L: q999 {q:.2e} max {m:.2e}")
    assert q <= 5e-4 and m <= 5e-3, (q, m)
    loss, dW, dth = gpu_ctx.lista_grad(d["K"], d["W"], d["th"], d["Y"], d["Xt"])
    le, dWe, dthe = OL.backward(K64, Wp, th, Y, X, rounded=True)
    print(f"loss {loss:.6e} model {le:.6e}")
    assert abs(loss - le) <= 1e-5 * le
    for l in range(L):
        g = dW[l].double().cpu().numpy()
        q, m = entrywise(g, dWe[l])
        fro = np.linalg.norm(g - dWe[l]) / np.linalg.norm(dWe[l])
        print(f"dW[{l}]: q999 {q:.2e} max {m:.2e} fro {fro:.2e}")
        assert q <= 3e-3 and m <= 1e-1 and fro <= 5e-3, (l, q, m, fro)
    t = dth.double().cpu().numpy()
    print("dtheta", t, dthe)
    assert np.all(np.abs(t - dthe) <= 1e-3 * np.abs(dthe).max())


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
