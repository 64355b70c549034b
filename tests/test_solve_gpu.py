"""gpl1_solve (Alg. GP + SS on eq. 2) on the GPU against the FP64 oracle.

Bars (from the method's own numbers, not tuned to the kernel):
  * relative objective gap (f(x_gpu) - f*) / f* <= 1e-6, with f(x_gpu) evaluated
    in FP64 by the oracle on the returned x and f* from the oracle run to its
    precision floor (stored for the full-size workloads in tests/golden/);
  * ||x_gpu - x*|| / ||x*|| <= 1e-4 where the problem's conditioning lets a
    1e-6 gap imply it (small Gaussian instances, FP64 config 0);
  * feasibility ||x||_1 <= rho (1 + 1e-6) and the sign conditions of the
    lambda-rho relation of Sec. 1 on the support.
"""
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
GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fstar.json")))


def to_dev(prob):
    if prob.dtype == W.DT_BF16:
        K = torch.from_numpy(prob.K.view(np.int16)).to(DEV)
    else:
        K = torch.from_numpy(prob.K).to(DEV)
    return K, torch.from_numpy(prob.y).to(DEV)


def gpu_solve(ctx, prob, x0=None, **kw):
    K, y = to_dev(prob)
    prm = pkg.params_default(**kw)
    x = None if x0 is None else torch.from_numpy(x0).to(DEV)
    x, res = ctx.solve(K, y, prob.rho, x=x, p=prob.p, params=prm)
    torch.cuda.synchronize()
    return x.double().cpu().numpy(), res


def rel_gap(prob, x, fstar):
    return (oracle.objective(prob, x) - fstar) / fstar


def small(n, p, k, dtype, seed, law="gauss", rho_scale=0.8, sigma=0.01):
    return W.gaussian(n, p, k, dtype=dtype, seed=seed, law=law, sigma=sigma, rho_scale=rho_scale)


ENGINES = [pytest.param(pkg.ENGINE_ONE_READ, id="one_read"), pytest.param(pkg.ENGINE_TWO_PASS, id="two_pass")]


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("dtype,n,p", [(W.DT_F32, 300, 1000), (W.DT_F32, 97, 301), (W.DT_F64, 256, 1024),
                                       (W.DT_BF16, 300, 1200), (W.DT_F32, 1000, 5000), (W.DT_BF16, 61, 257)])
def test_small_vs_oracle(gpu_ctx, dtype, n, p, engine):
    prob = small(n, p, max(3, n // 20), dtype, seed=n * 7 + p)
    xs, rs, _ = oracle.reference_solve(prob)
    x, res = gpu_solve(gpu_ctx, prob, stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, f_star=rs.f, max_iter=20000,
                       engine=engine)
    assert res.status == 0, res.as_dict()
    gap = rel_gap(prob, x, rs.f)
    assert gap <= 1e-6, gap
    assert np.abs(x).sum() <= prob.rho * (1 + 1e-6)
    err = np.linalg.norm(x - xs) / np.linalg.norm(xs)
    assert err <= 1e-3, err      # a 5e-7 gap on these well-conditioned instances


def test_config0_fp64_parity(gpu_ctx):
    prob = W.config0()
    fstar = GOLDEN["c0"]["f_star"]
    xs, rs, _ = oracle.reference_solve(prob)
    x, res = gpu_solve(gpu_ctx, prob, stop_rule=pkg.STOP_ON_REL_GAP, tol=1e-6, f_star=fstar)
    assert res.status == 0 and res.stop == 0, res.as_dict()
    assert rel_gap(prob, x, fstar) <= 1e-6
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-4
    # tighter stop: the FP64 path follows the oracle much further
    x, res = gpu_solve(gpu_ctx, prob, stop_rule=pkg.STOP_ON_REL_GAP, tol=1e-12, f_star=fstar, max_iter=5000)
    assert rel_gap(prob, x, fstar) <= 1e-11
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-6


@pytest.mark.parametrize("engine", ENGINES)
def test_config0_trace_matches_oracle_early(gpu_ctx, engine):
    """FP64: the first iterations take the same steps as the oracle (same alpha, lambda)."""
    prob = W.config0()
    for iters in (1, 2, 5, 10):
        x, res = gpu_solve(gpu_ctx, prob, stop_rule=0, max_iter=iters, engine=engine)
        xo, ro, tr = oracle.gpss(prob, trace=True, tol=0.0, max_iter=iters)
        assert res.iters == iters and res.status == 3
        np.testing.assert_allclose(x, xo, rtol=0, atol=1e-10 * np.abs(xo).max())
        assert abs(res.alpha - tr[-1, 1]) <= 1e-9 * tr[-1, 1]


def kkt_ok(prob, x, rel):
    f, lam, fw, g = oracle.certificates(prob, x)
    c = -0.5 * g
    supp = np.abs(x) > 1e-3 * np.abs(x).max()
    assert np.abs(x).sum() <= prob.rho * (1 + 1e-6)
    assert np.abs(x).sum() >= prob.rho * (1 - 1e-5)            # constraint active
    assert np.all(np.abs(c[supp] - lam * np.sign(x[supp])) <= rel * lam)
    return lam


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_full_size_configs(gpu_ctx, name):
    prob = W.config1() if name == "c1" else W.config2()
    gold = GOLDEN[name]
    x, res = gpu_solve(gpu_ctx, prob, stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, f_star=gold["f_star"],
                       max_iter=20000)
    gap = rel_gap(prob, x, gold["f_star"])
    assert res.status == 0, (res.as_dict(), gap)
    assert gap <= 1e-6, gap
    lam = kkt_ok(prob, x, rel=1e-2 if name == "c1" else 0.5)
    assert abs(lam - gold["lambda"]) <= 0.05 * gold["lambda"]


def test_orthonormal_closed_form(gpu_ctx):
    prob = W.orthonormal(600, 300, 20, seed=5, rho_scale=0.5)
    K = prob.K_f64()
    v = K.T @ prob.y
    xs, _ = oracle.project(v, prob.rho)        # x* = P(K^T y) for K^T K = I
    x, res = gpu_solve(gpu_ctx, prob, stop_rule=0, max_iter=2)
    np.testing.assert_allclose(x, xs, atol=1e-12 * np.abs(xs).max())


def test_infeasible_x0_is_projected(gpu_ctx):
    prob = small(300, 1000, 15, W.DT_F32, seed=44)
    _, rs, _ = oracle.reference_solve(prob)
    x0 = (np.random.default_rng(1).standard_normal(prob.p) * 10).astype(np.float32)   # ||x0||_1 >> rho
    x, res = gpu_solve(gpu_ctx, prob, x0=x0, stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, f_star=rs.f)
    assert res.status == 0
    assert rel_gap(prob, x, rs.f) <= 1e-6
    # one iteration from x0: equals the oracle's first iterate from the same x0
    x1, _ = gpu_solve(gpu_ctx, prob, x0=x0, stop_rule=0, max_iter=1)
    xo, _, _ = oracle.gpss(prob, x0=x0.astype(np.float64), tol=0.0, max_iter=1)
    np.testing.assert_allclose(x1, xo, rtol=0, atol=1e-4 * np.abs(xo).max())


def test_inactive_constraint_gives_least_squares(gpu_ctx):
    rng = np.random.default_rng(8)
    n, p = 400, 100
    K = rng.standard_normal((n, p)) / np.sqrt(n)
    y = rng.standard_normal(n)
    x_ls = np.linalg.lstsq(K, y, rcond=None)[0]
    prob = W.Problem(np.ascontiguousarray(K), n, p, p, W.DT_F64, y, 10 * np.abs(x_ls).sum(), x_ls, "ls")
    x, res = gpu_solve(gpu_ctx, prob, stop_rule=pkg.STOP_ON_REL_GAP, tol=1e-14,
                       f_star=np.sum((K @ x_ls - y) ** 2), max_iter=5000)
    # a 1e-14 relative gap on f* ~ 300 bounds ||K dx|| by 2e-6, so |dx| <~ 1e-5
    np.testing.assert_allclose(x, x_ls, atol=1e-5)


def test_degenerate_zero_data_and_tiny_shapes(gpu_ctx):
    # y = 0: x0 = 0 is optimal; the first projection returns x0 (stationary)
    prob = small(50, 80, 3, W.DT_F32, seed=2)
    prob.y[:] = 0
    x, res = gpu_solve(gpu_ctx, prob, stop_rule=0, max_iter=10)
    assert res.stop == 1 and res.iters == 0 and np.all(x == 0)
    # n = 1 and p = 1
    for n, p in [(1, 40), (30, 1), (1, 1)]:
        prob = small(n, p, 1, W.DT_F64, seed=n + p, rho_scale=0.5)
        xs, rs, _ = oracle.reference_solve(prob)
        x, res = gpu_solve(gpu_ctx, prob, stop_rule=pkg.STOP_ON_REL_GAP, tol=1e-10,
                           f_star=max(rs.f, 1e-300), max_iter=2000)
        assert oracle.objective(prob, x) <= rs.f * (1 + 1e-8) + 1e-14


def test_status_paths(gpu_ctx):
    prob = W.config0()
    x, res = gpu_solve(gpu_ctx, prob, stop_rule=0, max_iter=3)
    assert res.status == 3 and res.stop == 3 and res.iters == 3       # NOT_CONVERGED
    # FW certificate stop: the returned point satisfies its own certificate
    x, res = gpu_solve(gpu_ctx, prob, stop_rule=pkg.STOP_ON_FW, tol=1e-4)
    f, lam, fw, g = oracle.certificates(prob, x)
    assert res.stop == 2 and fw <= 1.1e-4 * (f - fw)
    K, y = to_dev(prob)
    with pytest.raises(pkg.Gpl1Error) as e:
        gpu_ctx.solve(K, y, -1.0)
    assert e.value.status == 1
    with pytest.raises(pkg.Gpl1Error) as e:          # misaligned K
        gpu_ctx.solve(K.view(-1)[1:1 + 255 * 1024].view(255, 1024), y[:255], 1.0)
    assert e.value.status == 1


def test_bounded_wait_reports_timeout(gpu_ctx):
    """A group barrier that can never complete ends the solve with TIMEOUT, and
    the context keeps working afterwards."""
    prob = W.config0()
    K, y = to_dev(prob)
    prm = pkg.params_default(debug=pkg.DEBUG_UNREACHABLE_BARRIER, timeout_ns=50_000_000)
    _, res = gpu_ctx.solve(K, y, prob.rho, params=prm)
    assert res.status == 6 and res.stop == 4
    x, res = gpu_solve(gpu_ctx, prob, stop_rule=pkg.STOP_ON_REL_GAP, tol=1e-6, f_star=GOLDEN["c0"]["f_star"])
    assert res.status == 0 and rel_gap(prob, x, GOLDEN["c0"]["f_star"]) <= 1e-6


@pytest.mark.parametrize("dtype,p", [(W.DT_F32, 16800), (W.DT_F64, 3840), (W.DT_BF16, 16800)])
def test_largest_p_the_kernel_stages(gpu_ctx, dtype, p):
    """p at the limit of the two-pass kernel's staged x/v vector in shared memory
    (35 x 480 float entries, 8 x 480 double entries), with a ragged last box of
    columns: solved by both engines; one column more is refused by the two-pass
    engine and solved by the one-read engine (default)."""
    prob = small(192, p, 12, dtype, seed=p + dtype, rho_scale=0.8)
    xs, rs, _ = oracle.reference_solve(prob)
    for engine in (pkg.ENGINE_TWO_PASS, pkg.ENGINE_AUTO):
        x, res = gpu_solve(gpu_ctx, prob, stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, f_star=rs.f, max_iter=20000,
                           engine=engine)
        assert res.status == 0, (engine, res.as_dict())
        assert rel_gap(prob, x, rs.f) <= 1e-6, engine
        assert np.abs(x).sum() <= prob.rho * (1 + 1e-6), engine
    # one column more than the two-pass staging holds is refused there, not run
    K, y = to_dev(small(8, p + 1, 1, dtype, seed=1))
    with pytest.raises(pkg.Gpl1Error) as e:
        gpu_ctx.solve(K, y, 1.0, params=pkg.params_default(engine=pkg.ENGINE_TWO_PASS))
    assert e.value.status == 7


# columns the one-read engine takes at most: 16 CTAs per cluster, each with
# four 16-byte chunks per thread of its 256 consumer threads
ONE_READ_MAX_P = {W.DT_F32: 16 * 4 * 256 * 4, W.DT_F64: 16 * 4 * 256 * 2, W.DT_BF16: 16 * 4 * 256 * 8}


@pytest.mark.parametrize("dtype,p", [(W.DT_F32, 24000), (W.DT_F64, 9000)])
def test_one_read_engine_beyond_the_two_pass_limit(gpu_ctx, dtype, p):
    """Past the two-pass limit (clusters of 12 or 6 CTAs for F32, 9 or 5 for
    F64, as the autotuner picks): the one-read engine reaches the oracle's
    optimum; past its own limit it refuses with GPL1_ERR_UNSUPPORTED."""
    prob = small(192, p, 16, dtype, seed=p + 7 * dtype, rho_scale=0.8)
    xs, rs, _ = oracle.reference_solve(prob)
    x, res = gpu_solve(gpu_ctx, prob, stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, f_star=rs.f, max_iter=20000,
                       engine=pkg.ENGINE_ONE_READ)
    assert res.status == 0, res.as_dict()
    assert rel_gap(prob, x, rs.f) <= 1e-6
    assert np.linalg.norm(x - xs) <= 1e-3 * np.linalg.norm(xs)
    big = ONE_READ_MAX_P[dtype] + 1
    K, y = to_dev(small(4, big, 1, dtype, seed=2))
    with pytest.raises(pkg.Gpl1Error) as e:
        gpu_ctx.solve(K, y, 1.0, params=pkg.params_default(engine=pkg.ENGINE_ONE_READ))
    assert e.value.status == 7


def test_nonmonotone_line_search_matches_oracle(gpu_ctx):
    """M = 10: the FP64 path takes the oracle's steps through the early iterations,
    and the FP32 path reaches the 1e-6 gap."""
    prob = W.config0()
    for iters in (3, 12):
        x, res = gpu_solve(gpu_ctx, prob, stop_rule=0, max_iter=iters, M=10)
        xo, ro, tr = oracle.gpss(prob, trace=True, tol=0.0, max_iter=iters, M=10)
        assert res.iters == iters
        np.testing.assert_allclose(x, xo, rtol=0, atol=1e-10 * np.abs(xo).max())
    prob = small(300, 1000, 15, W.DT_F32, seed=91)
    xs, rs, _ = oracle.reference_solve(prob)
    x, res = gpu_solve(gpu_ctx, prob, stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, f_star=rs.f, max_iter=20000, M=10)
    assert res.status == 0, res.as_dict()
    assert rel_gap(prob, x, rs.f) <= 1e-6


def test_engine_autotuner_picks_lists_and_agrees(gpu_ctx):
    """GPL1_ENGINE_AUTO times the admissible engines once per shape and keeps the
    fastest (gpl1_solve_tuned lists it); every engine, pinned, reaches the same
    optimum."""
    prob = small(1024, 8192, 40, W.DT_F32, seed=77)
    xs, rs, _ = oracle.reference_solve(prob)
    before = len(gpu_ctx.solve_tuned())
    x, res = gpu_solve(gpu_ctx, prob, stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, f_star=rs.f, max_iter=20000,
                       engine=pkg.ENGINE_AUTO)
    tuned = gpu_ctx.solve_tuned()
    assert len(tuned) == before + 1
    entry = [t for t in tuned if t["shape"] == (W.DT_F32, 1024, 8192, 0)][0]
    assert entry["engine"] in (pkg.ENGINE_TWO_PASS, pkg.ENGINE_ONE_READ_NCH2, pkg.ENGINE_ONE_READ_NCH4)
    assert entry["ms"] > 0
    assert res.status == 0 and rel_gap(prob, x, rs.f) <= 1e-6
    for eng in (pkg.ENGINE_TWO_PASS, pkg.ENGINE_ONE_READ_NCH2, pkg.ENGINE_ONE_READ_NCH4):
        x, res = gpu_solve(gpu_ctx, prob, stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, f_star=rs.f, max_iter=20000,
                           engine=eng)
        assert res.status == 0 and rel_gap(prob, x, rs.f) <= 1e-6, eng
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-3
    assert len(gpu_ctx.solve_tuned()) == before + 1   # pinned engines do not tune


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("name", ["c1", "c2"])
def test_fp32_trace_follows_the_fp64_oracle(gpu_ctx, name, engine):
    """FP32 data, full size: over the first 25 iterations the kernels take the
    oracle's decisions (the same Armijo steps lambda_k and Alg. SS ratio-test
    branches, so the same tau_k) and their steplengths alpha_k stay within 1e-3
    of the FP64 oracle's (measured: 2e-4), f_k within 1e-4.  Alg. SS and the
    line search run in FP64 on float-pair sums, so FP32 rounding enters only
    through the products with K."""
    prob = W.config1() if name == "c1" else W.config2()
    N = 25
    xo, ro, to = oracle.gpss(prob, trace=True, tol=0.0, max_iter=N)
    K, y = to_dev(prob)
    tr = torch.zeros(N, pkg.TRACE_COLS, dtype=torch.float64, device=DEV)
    prm = pkg.params_default(stop_rule=0, max_iter=N, engine=engine, x0_is_zero=1)
    _, res = gpu_ctx.solve(K, y, prob.rho, p=prob.p, params=prm, trace=tr)
    t = tr.cpu().numpy()
    assert res.iters == N
    np.testing.assert_array_equal(t[:, 2], to[:, 2])                    # lambda_k
    np.testing.assert_allclose(t[:, 3], to[:, 3], rtol=1e-6, atol=0)    # tau_k of Alg. SS
    np.testing.assert_allclose(t[:, 1], to[:, 1], rtol=1e-3, atol=0)    # alpha_k
    np.testing.assert_allclose(t[:, 0], to[:, 0], rtol=1e-4, atol=0)    # f(x_k)
