"""gpl1_solve_batched: many independent instances of uneven n, p in one
persistent launch, each checked against the FP64 oracle at the same bars as
single solves (relative objective gap <= 1e-6, feasibility)."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import paper_0902_4424_gb300 as pkg
import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def upload(prob):
    if prob.dtype == W.DT_BF16:
        K = torch.from_numpy(prob.K.view(np.int16)).to(DEV)
    else:
        K = torch.from_numpy(prob.K).to(DEV)
    y = torch.from_numpy(prob.y).to(DEV)
    x = torch.zeros(prob.p, dtype=torch.float64 if prob.dtype == W.DT_F64 else torch.float32, device=DEV)
    return K, y, x


def run_batch(ctx, probs, dtype, fstars, tol=5e-7):
    keep, descs = [], []
    for pr, fs in zip(probs, fstars):
        K, y, x = upload(pr)
        keep.append((K, y, x))
        descs.append(pkg.Context.make_problem(K, y, pr.rho, x, pr.p, fs))
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=tol, x0_is_zero=1, max_iter=20000)
    res = ctx.solve_batched(descs, dtype, prm)
    torch.cuda.synchronize()
    return [k[2].double().cpu().numpy() for k in keep], res


@pytest.mark.parametrize("dtype", [W.DT_BF16, W.DT_F32])
def test_ragged_batch_vs_oracle(gpu_ctx, dtype):
    rng = np.random.default_rng(17)
    sizes = [int(v) for v in rng.integers(16, 420, size=40)]
    sizes[:4] = [1, 2, 31, 419]                     # degenerate and ragged rows
    probs = [W.gaussian(n, 4 * n, max(1, n // 20), dtype=dtype, seed=1000 + i, law="pm1")
             for i, n in enumerate(sizes)]
    refs = [oracle.reference_solve(p)[1].f for p in probs]
    xs, res = run_batch(gpu_ctx, probs, dtype, refs)
    for pr, x, r, fs in zip(probs, xs, res, refs):
        f = oracle.objective(pr, x)
        assert r.status == 0, (pr.n, r.as_dict(), f, fs)
        assert (f - fs) <= 1e-6 * fs + 1e-12, (pr.n, f, fs)
        assert np.abs(x).sum() <= pr.rho * (1 + 1e-6)


def test_ragged_batch_config3_shapes(gpu_ctx):
    """Instances drawn like the 512-instance ragged batch (n in [128, 2048],
    p = 4n, BF16 K, +-1 signals with n/20 non-zeros): the first 16 of them,
    each against the oracle's optimum."""
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c3a_fstar.json")))
    sizes = gold["n"][:16]
    probs = [W.ragged_instance(i, n) for i, n in enumerate(sizes)]
    refs = gold["f_star"][:16]
    xs, res = run_batch(gpu_ctx, probs, W.DT_BF16, refs)
    for pr, x, r, fs in zip(probs, xs, res, refs):
        gap = (oracle.objective(pr, x) - fs) / fs
        assert r.status == 0 and r.stop == 0, (pr.n, r.as_dict(), gap)
        assert gap <= 1e-6
        assert np.abs(x).sum() <= pr.rho * (1 + 1e-6)


def test_batched_plan_replays_the_batched_solve(gpu_ctx):
    """gpl1_plan_*: the batched solve recorded as a CUDA graph gives, on every replay,
    the iterates and results of gpl1_solve_batched (the same kernel on the same
    instances), and follows right-hand sides rewritten in place between replays."""
    rng = np.random.default_rng(5)
    sizes = [int(v) for v in rng.integers(32, 300, size=12)]
    probs = [W.gaussian(n, 4 * n, max(1, n // 20), dtype=W.DT_F32, seed=2000 + i, law="pm1")
             for i, n in enumerate(sizes)]
    keep = [upload(pr) for pr in probs]
    descs = [pkg.Context.make_problem(K, y, pr.rho, x, pr.p) for (K, y, x), pr in zip(keep, probs)]
    prm = pkg.params_default(stop_rule=0, x0_is_zero=1, max_iter=40)
    ref = gpu_ctx.solve_batched(descs, W.DT_F32, prm)
    torch.cuda.synchronize()
    x_ref = [x.clone() for _, _, x in keep]
    plan = gpu_ctx.plan_batched(descs, W.DT_F32, prm)
    for _ in range(2):
        for _, _, x in keep:
            x.fill_(7.0)                                 # x0 = 0 is re-established by the graph
        res = plan.run()
        torch.cuda.synchronize()
        for (_, _, x), xr, r, rr in zip(keep, x_ref, res, ref):
            assert torch.equal(x, xr)
            assert (r.status, r.iters, r.f, r.backtracks) == (rr.status, rr.iters, rr.f, rr.backtracks)
    # new right-hand sides in place: the replay solves them
    for (_, y, _), pr in zip(keep, probs):
        y.mul_(0.5)
    res = plan.run()
    torch.cuda.synchronize()
    x_new = [x.clone() for _, _, x in keep]
    ref2 = gpu_ctx.solve_batched(descs, W.DT_F32, prm)
    torch.cuda.synchronize()
    for (_, _, x), xn, r, rr in zip(keep, x_new, res, ref2):
        assert torch.equal(x, xn)
        assert (r.status, r.iters, r.f) == (rr.status, rr.iters, rr.f)
    plan.close()


def test_async_solves_match_the_synchronous_ones(gpu_ctx):
    """gpl1_solve_batched_async / gpl1_solve_async: enqueued without waiting, results
    in device memory, the same iterates and results as the synchronous calls; the
    stream orders two asynchronous solves on one context."""
    import ctypes
    rng = np.random.default_rng(9)
    sizes = [int(v) for v in rng.integers(40, 260, size=6)]
    probs = [W.gaussian(n, 4 * n, max(1, n // 20), dtype=W.DT_F32, seed=3000 + i, law="pm1")
             for i, n in enumerate(sizes)]
    keep = [upload(pr) for pr in probs]
    descs = [pkg.Context.make_problem(K, y, pr.rho, x, pr.p) for (K, y, x), pr in zip(keep, probs)]
    prm = pkg.params_default(stop_rule=0, x0_is_zero=1, max_iter=30)
    ref = gpu_ctx.solve_batched(descs, W.DT_F32, prm)
    torch.cuda.synchronize()
    x_ref = [x.clone() for _, _, x in keep]
    for _, _, x in keep:
        x.fill_(5.0)
    r1 = gpu_ctx.solve_batched_async(descs, W.DT_F32, prm)
    x_mid = [x.clone() for _, _, x in keep]      # stream-ordered after the first solve
    r2 = gpu_ctx.solve_batched_async(descs, W.DT_F32, prm)
    torch.cuda.synchronize()
    for res in (r1, r2):
        got = pkg.Context.results_from_device(res, len(descs))
        for g, rr in zip(got, ref):
            assert (g.status, g.iters, g.f, g.backtracks) == (rr.status, rr.iters, rr.f, rr.backtracks)
    for (_, _, x), xm, xr in zip(keep, x_mid, x_ref):
        assert torch.equal(x, xr) and torch.equal(xm, xr)
    # the single-instance form (a multi-CTA solve, which agrees with another run to
    # rounding only): solved to the oracle gap through the asynchronous call
    K, y, x = keep[0]
    fs = oracle.reference_solve(probs[0])[1].f
    prm_gap = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, x0_is_zero=1, max_iter=20000)
    res = torch.empty(ctypes.sizeof(pkg.Result), dtype=torch.uint8, device=DEV)
    pr = pkg.Context.make_problem(K, y, probs[0].rho, x, probs[0].p, fs)
    st = pkg.lib().gpl1_solve_async(gpu_ctx._h, ctypes.byref(pr), W.DT_F32, ctypes.byref(prm_gap),
                                    ctypes.c_void_p(res.data_ptr()))
    assert st == 0
    torch.cuda.synchronize()
    g = pkg.Context.results_from_device(res, 1)[0]
    assert g.status == 0 and g.stop == 0, g.as_dict()
    assert (oracle.objective(probs[0], x.double().cpu().numpy()) - fs) / fs <= 1e-6


def test_plan_of_a_single_instance(gpu_ctx):
    """A plan of one instance records the multi-CTA cooperative launch of the single
    solve; every replay solves the instance to the oracle gap, as gpl1_solve does (the
    two agree to rounding, not bit for bit: the multi-CTA solve adds partial products
    with float atomics)."""
    prob = W.gaussian(300, 1200, 15, dtype=W.DT_F32, seed=77, law="pm1")
    fs = oracle.reference_solve(prob)[1].f
    K, y, x = upload(prob)
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, x0_is_zero=1, max_iter=20000)
    x1, r1 = gpu_ctx.solve(K, y, prob.rho, x=x.clone(), p=prob.p, params=prm, f_star=fs)
    torch.cuda.synchronize()
    assert r1.status == 0
    plan = gpu_ctx.plan_batched([pkg.Context.make_problem(K, y, prob.rho, x, prob.p, fs)], W.DT_F32, prm)
    for _ in range(2):
        x.fill_(1.0)   # x0 = 0 is re-established by the graph
        (r,) = plan.run()
        torch.cuda.synchronize()
        assert r.status == 0 and r.stop == 0, r.as_dict()
        assert (oracle.objective(prob, x.double().cpu().numpy()) - fs) / fs <= 1e-6
    plan.close()


def test_batched_degenerate_instances(gpu_ctx):
    """A batch (FP64) mixing the degenerate cases with ordinary ones: y = 0 (x0 = 0 is
    stationary at once), a radius above ||x_LS||_1 (the constraint inactive: the
    least-squares solution), n = 1, and two ordinary instances."""
    rng = np.random.default_rng(21)
    probs, fstars = [], []
    zero = W.gaussian(40, 160, 4, dtype=W.DT_F64, seed=31)
    zero.y[:] = 0.0
    probs.append(zero)
    fstars.append(0.0)
    n, p = 120, 40                                  # inactive constraint
    K = rng.standard_normal((n, p)) / np.sqrt(n)
    y = rng.standard_normal(n)
    x_ls = np.linalg.lstsq(K, y, rcond=None)[0]
    probs.append(W.Problem(np.ascontiguousarray(K), n, p, p, W.DT_F64, y, 10 * np.abs(x_ls).sum(), x_ls, "ls"))
    fstars.append(float(np.sum((K @ x_ls - y) ** 2)))
    for pr in (W.gaussian(1, 40, 1, dtype=W.DT_F64, seed=32, rho_scale=0.5),
               W.gaussian(60, 240, 6, dtype=W.DT_F64, seed=33), W.gaussian(200, 800, 10, dtype=W.DT_F64, seed=34)):
        probs.append(pr)
        fstars.append(oracle.reference_solve(pr)[1].f)
    keep = [upload(pr) for pr in probs]
    descs = [pkg.Context.make_problem(Kd, yd, pr.rho, x, pr.p, fs if fs > 0 else -1.0)
             for (Kd, yd, x), pr, fs in zip(keep, probs, fstars)]
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=1e-10, x0_is_zero=1, max_iter=100000)
    res = gpu_ctx.solve_batched(descs, W.DT_F64, prm)
    torch.cuda.synchronize()
    xs = [x.double().cpu().numpy() for _, _, x in keep]
    assert res[0].stop == 1 and res[0].iters == 0 and np.all(xs[0] == 0)          # stationary at x0 = 0
    assert res[1].status == 0
    # least squares: a 1e-10 gap on f* bounds ||K dx|| by about 1e-4, so |dx| <~ 3e-4
    np.testing.assert_allclose(xs[1], x_ls, atol=1e-3)
    # n = 1 fits y almost exactly (f* ~ 0): the relative-gap stop may not be reachable and
    # the instance runs to max_iter (status 3); its objective is checked all the same
    for q in (2, 3, 4):
        assert res[q].status in (0, 3), (q, res[q].as_dict())
        f = oracle.objective(probs[q], xs[q])
        bar = 1e-8 if q == 2 else 1e-6
        assert f - fstars[q] <= bar * fstars[q] + 1e-14, q
        assert np.abs(xs[q]).sum() <= probs[q].rho * (1 + 1e-9)
