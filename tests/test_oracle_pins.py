"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each check below would fail for a plausible slip in the oracle: a dropped
factor 2 in the gradient, a swapped BB rule, a wrong direction of the ratio
test or of the tau update, an off-by-one in the sorted projection, a sign
error in the soft threshold, an Armijo test with the wrong sign.

* Projection onto the l1 ball (the paper uses P_Omega without giving an
  algorithm): brute force over supports and signs, identity inside the ball,
  l1 norm equal to rho on the boundary, soft-threshold form with a threshold
  found by bisection, the variational inequality of a Euclidean projection.
* Algorithm GP + SS on eq. 2:
    - the closed form for K with orthonormal columns (the solution is the
      projection of K^T y), reached by the first BB step, which equals 1/2;
    - brute force over supports and signs for tiny p (n >= p);
    - the equivalence of eq. 1 and eq. 2 and the lambda-rho relation of Sec. 1,
      checked with FISTA (eq. fista), an independent algorithm for eq. 1;
    - the KKT sign conditions on the configurations;
    - a 3-iteration trace on a diagonal problem derived by hand (below);
    - monotone decrease (M = 1), feasibility, steplength bounds.
* The comparison methods of Sec. 2 (oracle/methods.py): ISTA/FISTA and PSD in
  one step on an orthonormal K (closed forms of eq. 1 and eq. 2), a PSD step
  on a diagonal K derived by hand, FISTA's first step and momentum weight, and
  all three at the exact homotopy points.
* The learned warm start (oracle/lista.py) and the homotopy path
  (oracle/homotopy.py): see their sections below.
"""
import itertools
import json
import sys
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import methods

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
sys.path.insert(0, GOLDEN)


# ----------------------------------------------------------------- helpers

def brute_project(v, rho):
    """min ||w - v||^2 over ||w||_1 <= rho by enumerating sign patterns sigma in {-1,0,1}^p.

    For a fixed sign pattern with support S the minimiser on the face
    sigma^T w_S = rho is w_S = v_S - ((sigma^T v_S - rho)/|S|) sigma; it is a
    candidate when its signs agree with sigma.
    """
    v = np.asarray(v, float)
    if np.abs(v).sum() <= rho:
        return v.copy()
    best, best_w = np.inf, None
    for sig in itertools.product((-1, 0, 1), repeat=v.size):
        sig = np.array(sig, float)
        S = sig != 0
        if not S.any():
            continue
        w = np.zeros_like(v)
        w[S] = v[S] - (sig[S] @ v[S] - rho) / S.sum() * sig[S]
        if np.any(sig[S] * w[S] < -1e-12):
            continue
        dist = ((w - v) ** 2).sum()
        if dist < best:
            best, best_w = dist, w
    return best_w


def soft_threshold_bisect(v, rho):
    """tau with sum(max(|v|-tau, 0)) = rho found by plain bisection."""
    a = np.abs(v)
    lo, hi = 0.0, a.max()
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.maximum(a - mid, 0).sum() > rho:
            lo = mid
        else:
            hi = mid
    tau = 0.5 * (lo + hi)
    return np.sign(v) * np.maximum(a - tau, 0), tau


def brute_eq2(K, y, rho):
    """min ||Kx - y||^2 s.t. ||x||_1 <= rho by enumerating supports and signs (n >= p).

    Candidates: for every support S the unconstrained least-squares solution
    (kept if ||x||_1 <= rho) and, for every sign vector sigma on S, the
    least-squares solution on the face sigma^T x_S = rho (kept if its signs
    agree with sigma).  The optimum is one of the candidates.
    """
    n, p = K.shape
    best, best_x = np.sum(y ** 2), np.zeros(p)
    for sig in itertools.product((-1, 0, 1), repeat=p):
        sig = np.array(sig, float)
        S = np.flatnonzero(sig)
        if S.size == 0:
            continue
        KS = K[:, S]
        A = KS.T @ KS
        b = KS.T @ y
        # face: [2A  s; s^T 0] [x; mu] = [2b; rho]
        M = np.zeros((S.size + 1, S.size + 1))
        M[:-1, :-1] = 2 * A
        M[:-1, -1] = sig[S]
        M[-1, :-1] = sig[S]
        rhs = np.concatenate([2 * b, [rho]])
        sol = np.linalg.solve(M, rhs)
        xs = sol[:-1]
        cands = []
        if np.all(sig[S] * xs >= -1e-12):
            cands.append(xs)
        xu = np.linalg.solve(A, b)
        if np.abs(xu).sum() <= rho:
            cands.append(xu)
        for c in cands:
            x = np.zeros(p)
            x[S] = c
            f = np.sum((K @ x - y) ** 2)
            if f < best:
                best, best_x = f, x
    return best_x, best


def fista(K, y, lam, iters):
    """FISTA (eq. fista) for min ||Kx - y||^2 + 2 lam ||x||_1 with step 1/||K||^2
    (oracle/methods.py; with ||K|| = 1 the paper's iteration itself)."""
    return methods.ista(K, y, lam, iters, step=1.0 / np.linalg.norm(K, 2) ** 2, fista=True)[0]


def dense_problem(K, y, rho):
    K = np.asarray(K, float)
    return W.Problem(np.ascontiguousarray(K), K.shape[0], K.shape[1], K.shape[1], W.DT_F64,
                     np.asarray(y, float), float(rho), np.zeros(K.shape[1]), "dense")


# --------------------------------------------------------------- projection

def test_project_identity_inside_ball():
    rng = np.random.default_rng(1)
    v = rng.standard_normal(257)
    w, tau = oracle.project(v, np.abs(v).sum() * 1.0001)
    assert tau == 0.0
    assert np.array_equal(w, v)
    w, tau = oracle.project(v, np.abs(v).sum())          # exactly on the boundary
    assert np.array_equal(w, v)


@pytest.mark.parametrize("seed", range(12))
def test_project_brute_force_tiny(seed):
    rng = np.random.default_rng(100 + seed)
    p = int(rng.integers(1, 8))
    v = rng.standard_normal(p) * rng.choice([0.1, 1, 10])
    if seed % 3 == 0:
        v[rng.integers(0, p)] = 0.0                      # sgn(0) = 0
    if seed % 4 == 1 and p > 1:
        v[1] = -v[0]                                     # tie in |v|
    rho = float(rng.uniform(0.05, 1.2) * np.abs(v).sum())
    w, _ = oracle.project(v, rho)
    np.testing.assert_allclose(w, brute_project(v, rho), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("p,scale", [(1000, 0.3), (4096, 0.01), (333, 0.9)])
def test_project_boundary_soft_threshold(p, scale):
    rng = np.random.default_rng(p)
    v = rng.standard_normal(p) * np.exp(rng.standard_normal(p))
    rho = scale * np.abs(v).sum()
    w, tau = oracle.project(v, rho)
    assert tau > 0
    assert abs(np.abs(w).sum() - rho) <= 1e-12 * rho
    assert np.all(w * v >= 0) and np.all(np.abs(w) <= np.abs(v))
    wb, taub = soft_threshold_bisect(v, rho)
    assert abs(tau - taub) <= 1e-12 * max(1.0, taub)
    np.testing.assert_allclose(w, wb, rtol=0, atol=1e-11 * np.abs(v).max())


def test_project_variational_inequality():
    rng = np.random.default_rng(7)
    v = rng.standard_normal(64) * 3
    rho = 5.0
    w, _ = oracle.project(v, rho)
    for _ in range(200):
        u = rng.standard_normal(64)
        u *= rng.uniform(0, 1) * rho / np.abs(u).sum()   # a point of the ball
        assert (v - w) @ (u - w) <= 1e-10


# --------------------------------------------------------------- GP + SS

def test_hand_derived_trace_diagonal():
    """K = diag(1, 3), y = (9, 1), rho = 100 (constraint inactive), x0 = 0.

    f(x) = (x1 - 9)^2 + (3 x2 - 1)^2,  grad f = (2 x1 - 18, 18 x2 - 6).
    k=0: g0 = (-18,-6); P(x0 - g0) = (18, 6) so alpha_0 = 1/18; h = (1, 1/3);
         f(h) = 64 <= 82 - 2e-3, lambda = 1; x1 = (1, 1/3).
    k=1: g1 = (-16, 0); s = (1, 1/3), z = (2, 6): s's = 10/9, s'z = 4, z'z = 40;
         BB1 = 5/18, BB2 = 1/10, ratio 0.36 <= tau_1 = 0.5 -> alpha_1 = min{a2_1}
         = 1/10 and tau_2 = 0.45; h = (2.6, 1/3), f = 40.96, lambda = 1.
    k=2: g2 = (-12.8, 0); s = (1.6, 0), z = (3.2, 0): BB1 = BB2 = 1/2, ratio 1 >
         0.45 -> alpha_2 = 1/2, tau_3 = 0.495; h = (9, 1/3) is the minimiser.
    """
    prob = dense_problem(np.diag([1.0, 3.0]), [9.0, 1.0], 100.0)
    x, res, tr = oracle.gpss(prob, trace=True, tol=0.0, max_iter=10)
    expect = np.array([[82.0, 1 / 18, 1.0, 0.5],
                       [64.0, 0.1, 1.0, 0.45],
                       [40.96, 0.5, 1.0, 0.495]])
    np.testing.assert_allclose(tr[:3], expect, rtol=1e-12)
    np.testing.assert_allclose(x, [9.0, 1 / 3], rtol=1e-12)


def test_orthonormal_closed_form():
    """K^T K = I: f(x) = ||x - K^T y||^2 + const, so x* = P(K^T y) = S_tau(K^T y).

    From x0 = 0 the BB steps at k = 1 are both 1/2 (s^T z = 2 s^T s), which
    sends x_1 - alpha_1 g_1 to K^T y exactly, so x_2 = P(K^T y).  (Further
    iterations only move x by rounding noise.)
    """
    prob = W.orthonormal(300, 120, 15, seed=3, rho_scale=0.5)
    K = prob.K_f64()
    xs, tau = soft_threshold_bisect(K.T @ prob.y, prob.rho)
    x, res, tr = oracle.gpss(prob, trace=True, tol=0.0, max_iter=2)
    np.testing.assert_allclose(x, xs, atol=1e-12 * np.abs(xs).max())
    assert abs(tr[1, 1] - 0.5) < 1e-12 and tr[1, 2] == 1.0
    f, lam, fw, g = oracle.certificates(prob, x)
    assert abs(lam - tau) <= 1e-9 * tau          # lambda = max|K^T(y - Kx)| = tau here
    assert abs(f - np.sum((K @ xs - prob.y) ** 2)) <= 1e-10 * f


@pytest.mark.parametrize("seed", range(6))
def test_gpss_brute_force_tiny(seed):
    rng = np.random.default_rng(500 + seed)
    p = int(rng.integers(2, 7))
    n = p + int(rng.integers(0, 4))
    K = rng.standard_normal((n, p))
    y = rng.standard_normal(n)
    x_ls = np.linalg.lstsq(K, y, rcond=None)[0]
    rho = float(rng.uniform(0.1, 1.3) * np.abs(x_ls).sum())
    xb, fb = brute_eq2(K, y, rho)
    x, res, _ = oracle.reference_solve(dense_problem(K, y, rho))
    assert res.f <= fb * (1 + 1e-12) + 1e-14
    np.testing.assert_allclose(x, xb, atol=1e-7 * max(1, np.abs(xb).max()))


def test_lambda_rho_relation_fista():
    """Eq. 1 at lambda and eq. 2 at rho = ||xbar(lambda)||_1 have the same minimiser,
    and lambda = max|K^T(y - K x~(rho))| (Sec. 1)."""
    rng = np.random.default_rng(11)
    n, p = 60, 150
    K = rng.standard_normal((n, p)) / np.sqrt(n)
    x0 = np.zeros(p)
    x0[rng.permutation(p)[:8]] = rng.standard_normal(8)
    y = K @ x0 + 0.01 * rng.standard_normal(n)
    lam_max = np.abs(K.T @ y).max()
    lam = lam_max / 6
    xbar = fista(K, y, lam, 30000)
    rho = np.abs(xbar).sum()
    x, res, _ = oracle.reference_solve(dense_problem(K, y, rho))
    np.testing.assert_allclose(x, xbar, atol=1e-7)
    assert abs(res.lambda_reg - lam) <= 1e-6 * lam


def test_lambda_max_zero_solution():
    """xbar(lambda) = 0 for lambda >= lambda_max = max|K^T y| (Sec. 1)."""
    rng = np.random.default_rng(12)
    K = rng.standard_normal((30, 50)) / np.sqrt(30)
    y = rng.standard_normal(30)
    lam_max = np.abs(K.T @ y).max()
    assert np.all(fista(K, y, lam_max * 1.0001, 500) == 0)
    # on the eq. 2 side: rho -> 0 gives lambda -> lambda_max
    x, res, _ = oracle.reference_solve(dense_problem(K, y, 1e-9))
    assert abs(res.lambda_reg - lam_max) <= 1e-6 * lam_max


def kkt_check(prob, x, rel=1e-6):
    f, lam, fw, g = oracle.certificates(prob, x)
    c = -0.5 * g                                  # c = K^T (y - K x)
    supp = np.abs(x) > 1e-9 * np.abs(x).max()
    assert abs(np.abs(x).sum() - prob.rho) <= 1e-9 * prob.rho       # constraint active
    assert np.all(np.abs(c[supp] - lam * np.sign(x[supp])) <= rel * lam)
    assert np.all(np.abs(c) <= lam * (1 + 1e-12))
    return f, lam


def test_config0_kkt_and_invariants():
    prob = W.config0()
    x, res, _ = oracle.reference_solve(prob)
    kkt_check(prob, x)
    # invariants of a 1e-6 run: monotone f (M = 1), feasibility, alpha in range,
    # tau changed only by 0.9 or 1.1, lambda a power of theta
    x6, r6, tr = oracle.gpss(prob, trace=True, f_star=res.f, tol=1e-6)
    assert r6.stop == 0 and (r6.f - res.f) <= 1e-6 * res.f
    assert np.all(np.diff(tr[:, 0]) <= 0)
    assert np.all((tr[:, 1] >= 1e-10) & (tr[:, 1] <= 1e10))
    ratios = tr[1:, 3] / tr[:-1, 3]
    assert np.all(np.isclose(ratios, 0.9) | np.isclose(ratios, 1.1) | np.isclose(ratios, 1.0))
    assert np.all(np.isclose(np.log2(tr[:, 2]), np.round(np.log2(tr[:, 2]))))
    assert np.abs(x6).sum() <= prob.rho * (1 + 1e-12)


def test_golden_fstar_values_match_oracle_small():
    """The stored f* of config 0 was written by tests/golden/make_golden.py from the oracle."""
    with open(os.path.join(GOLDEN, "fstar.json")) as fh:
        gold = json.load(fh)
    prob = W.config0()
    x, res, _ = oracle.reference_solve(prob)
    assert abs(res.f - gold["c0"]["f_star"]) <= 1e-12 * res.f


def test_golden_c3a_fstar_match_oracle():
    """The stored optima of the ragged batch are the oracle's: recompute the two smallest."""
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c3a_fstar.json")))
    assert gold["n"] == W.ragged_sizes(len(gold["n"]))
    order = np.argsort(gold["n"])[:2]
    for i in order:
        prob = W.ragged_instance(int(i), gold["n"][i])
        f = oracle.floor_solve(prob)[1].f
        assert abs(f - gold["f_star"][i]) <= 1e-12 * gold["f_star"][i]


def test_golden_c5_fstar_match_oracle_and_the_path():
    """The stored optima of the radius sweep are the oracle's (recompute the smallest
    radius), and they trace the solution path: f* falls as rho grows (a larger
    ball), convex in rho (the value function of a convex problem in its radius),
    and at rho = ||x_true||_1 it sits near the noise level."""
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c5_fstar.json")))
    Ks, ldk, n, y, rho, xt = W.rho_sweep()
    assert np.allclose(gold["rho"], rho, rtol=1e-15)
    prob = W.Problem(Ks, n, xt.shape[0], ldk, W.DT_BF16, y.copy(), float(rho[0]), xt, "c5_0")
    f0 = oracle.floor_solve(prob)[1].f
    assert abs(f0 - gold["f_star"][0]) <= 1e-12 * f0
    f = np.array(gold["f_star"])
    assert np.all(np.diff(f) < 0)
    slope = np.diff(f) / np.diff(rho)
    assert np.all(np.diff(slope) >= -1e-9 * np.abs(slope[:-1]))
    K = W.bf16_bits_to_f64(Ks[:, :xt.shape[0]])
    noise2 = float(np.sum((y.astype(np.float64) - K @ xt) ** 2))
    assert 0.2 * noise2 <= f[-1] <= noise2


# ------------------------------------------------------- learned warm start
from oracle import lista  # noqa: E402


def eq1_optimality_residual(K, y, x, lam):
    """How far x is from the optimality conditions of eq. 1 (min ||Kx-y||^2 + 2 lam ||x||_1):
    c = K^T (y - K x) must equal lam sgn(x) on the support and satisfy |c| <= lam off it."""
    c = K.T @ (y - K @ x)
    on = x != 0
    r_on = np.max(np.abs(c[on] - lam * np.sign(x[on]))) if on.any() else 0.0
    r_off = max(0.0, np.max(np.abs(c[~on])) - lam) if (~on).any() else 0.0
    return max(r_on, r_off)


def test_lista_one_layer_on_orthonormal_k_solves_eq1():
    rng = np.random.default_rng(31)
    n, p = 40, 16
    K, _ = np.linalg.qr(rng.standard_normal((n, p)))
    y = rng.standard_normal((3, n))
    lam = 0.3
    xs, _ = lista.forward(K, K.T[None], np.array([lam]), y)
    for b in range(3):
        assert eq1_optimality_residual(K, y[b], xs[1][b], lam) <= 1e-12


def test_lista_tied_ista_layers_reach_eq1_optimality():
    rng = np.random.default_rng(32)
    n, p = 30, 60
    K = rng.standard_normal((n, p)) / np.sqrt(n)
    y = rng.standard_normal((2, n))
    lam = 0.2
    W, theta, Lk = lista.init_params(K, 1, lam)
    assert abs(Lk - np.linalg.norm(K, 2) ** 2) <= 1e-6 * Lk   # power iteration, 200 steps
    layers = 4000
    xs, _ = lista.forward(K, np.repeat(W, layers, axis=0), np.full(layers, theta[0]), y)
    # each layer is the proximal-gradient step of 1/2 ||Kx-y||^2 + lam ||x||_1 (step 1/L), whose
    # minimiser is eq. 1's at the same lam (both have K^T (y - Kx) in lam d||x||_1)
    for b in range(2):
        assert eq1_optimality_residual(K, y[b], xs[-1][b], lam) <= 1e-6


def test_lista_backward_matches_finite_differences():
    rng = np.random.default_rng(33)
    n, p, L, B = 6, 10, 3, 4
    K = rng.standard_normal((n, p)) / np.sqrt(n)
    Y = rng.standard_normal((B, n))
    Xt = rng.standard_normal((B, p)) * (rng.random((B, p)) < 0.3)
    W = rng.standard_normal((L, p, n)) * 0.3
    theta = np.array([0.05, 0.08, 0.03])
    f0, dW, dth = lista.backward(K, W, theta, Y, Xt)
    h = 1e-6
    for (l, i, j) in [(0, 0, 0), (1, 3, 2), (2, 9, 5), (0, 5, 4), (2, 1, 1)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[l, i, j] += h
        Wm[l, i, j] -= h
        fp = lista.loss(lista.forward(K, Wp, theta, Y)[0][-1], Xt)
        fm = lista.loss(lista.forward(K, Wm, theta, Y)[0][-1], Xt)
        assert abs((fp - fm) / (2 * h) - dW[l, i, j]) <= 1e-6 * max(1.0, abs(dW[l, i, j]))
    for l in range(L):
        tp, tm = theta.copy(), theta.copy()
        tp[l] += h
        tm[l] -= h
        fp = lista.loss(lista.forward(K, W, tp, Y)[0][-1], Xt)
        fm = lista.loss(lista.forward(K, W, tm, Y)[0][-1], Xt)
        assert abs((fp - fm) / (2 * h) - dth[l]) <= 1e-6 * max(1.0, abs(dth[l]))


def test_lista_bf16_rounding_is_round_to_nearest_even():
    """The precision model's rounding against torch's float32 -> bfloat16
    conversion (round to nearest, ties to even), bit for bit, including ties."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(41)
    a = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 6, 4000),
                        1.0 + np.arange(-8, 9) * 2.0 ** -8,            # ties at 1 + odd * 2^-8
                        1.0 + np.arange(-8, 9) * 2.0 ** -9])
    a = a.astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(lista.bf16(a), ref)
    assert lista.bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0                        # tie to even (down)
    assert lista.bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6        # tie to even (up)


def test_lista_precision_model_is_exact_on_representable_data():
    """With small sparse integers everywhere (every operand and every sum below
    2^8, so exactly representable in BF16 and FP32), the rounded network equals
    the FP64 network exactly, forward and backward: the model rounds only where
    a tensor-core implementation does, and never changes a representable value."""
    rng = np.random.default_rng(0)
    n, p, L, B = 4, 5, 2, 2
    K = rng.integers(-1, 2, (n, p)).astype(np.float64) * (rng.random((n, p)) < 0.6)
    W = rng.integers(-1, 2, (L, p, n)).astype(np.float64) * (rng.random((L, p, n)) < 0.6)
    Y = rng.integers(-3, 4, (B, n)).astype(np.float64)
    Xt = rng.integers(-2, 3, (B, p)).astype(np.float64)
    theta = np.array([1.0, 1.0])
    x64 = lista.forward(K, W, theta, Y)[0][-1]
    x16 = lista.forward(K, W, theta, Y, rounded=True)[0][-1]
    assert np.array_equal(x64, x16) and np.abs(x64).max() > 0
    l64, dW64, dt64 = lista.backward(K, W, theta, Y, Xt)
    l16, dW16, dt16 = lista.backward(K, W, theta, Y, Xt, rounded=True)
    assert np.abs(dW64).max() > 0 and np.count_nonzero(dt64) == L
    assert l64 == l16 and np.array_equal(dW64, dW16) and np.array_equal(dt64, dt16)


def test_lista_exact_case_loses_nothing_to_rounding():
    """The data of the kernels' exact LISTA test (workloads.lista_exact_case,
    K 64 x 128, batch 64, two layers): the BF16 precision model equals the FP64
    network exactly, forward and backward, with both layers active (between a
    third and a half of the pre-threshold values above theta) and every dW row
    touched.  Its values are multiples of 2^-10 below 2^8 in size (at most 18
    significant bits; the sums of the magnitudes of the terms of every product
    stay below 2^8 too, 173 at most for dtheta), so FP32 sums of them are exact
    in any order."""
    K, Wl, theta, Y, Xt = W.lista_exact_case()
    xs, zs = lista.forward(K, Wl, theta, Y)
    xr, _ = lista.forward(K, Wl, theta, Y, rounded=True)
    assert all(np.array_equal(a, b) for a, b in zip(xs, xr))
    for z, t in zip(zs, theta):
        assert 0.3 < np.mean(np.abs(z) > t) < 0.6
    l64, dW64, dt64 = lista.backward(K, Wl, theta, Y, Xt)
    l16, dW16, dt16 = lista.backward(K, Wl, theta, Y, Xt, rounded=True)
    assert l64 == l16 and np.array_equal(dW64, dW16) and np.array_equal(dt64, dt16)
    assert np.all(np.abs(dW64).max(axis=2) > 0)
    for v in (*xs, *zs, dW64, dt64):
        assert np.all(v * 2.0 ** 10 == np.round(v * 2.0 ** 10)) and np.abs(v).max() < 2.0 ** 8


def test_lista_precision_model_within_bf16_error_of_fp64():
    """On random data the rounded network differs from the FP64 one by about the
    BF16 unit roundoff (2^-9) compounded over the layers, and not by less than
    a rounding: the model does round."""
    rng = np.random.default_rng(43)
    n, p, L, B = 32, 96, 4, 8
    K = rng.standard_normal((n, p)) / np.sqrt(n)
    W0, th, _ = lista.init_params(K, L, 0.05)
    W = W0 * (1 + 0.2 * rng.standard_normal(W0.shape))
    Y = rng.standard_normal((B, n))
    x64 = lista.forward(K, W, th, Y)[0][-1]
    x16 = lista.forward(K, W, th, Y, rounded=True)[0][-1]
    rel = np.linalg.norm(x16 - x64) / np.linalg.norm(x64)
    assert 1e-5 < rel < 4 * L * 2.0 ** -9, rel


def test_nonmonotone_line_search_invariant():
    """M > 1 (the nonmonotone Armijo rule of Alg. GP, Step 4): every accepted value
    lies below the largest of the last M (gT d < 0), f need not decrease at every
    step, and the run reaches the same optimum as the monotone reference."""
    prob = W.config0()
    _, ref, _ = oracle.reference_solve(prob)
    M = 10
    x, r, tr = oracle.gpss(prob, trace=True, f_star=ref.f, tol=1e-6, M=M)
    assert r.stop == 0 and (r.f - ref.f) <= 1e-6 * ref.f
    f = tr[:, 0]
    for k in range(1, len(f)):
        assert f[k] < max(f[max(0, k - M):k]) or f[k] == f[k - 1] == 0.0
    assert np.abs(x).sum() <= prob.rho * (1 + 1e-12)


# ------------------------------------------------------- homotopy path (exact)
from oracle import homotopy  # noqa: E402


@pytest.mark.parametrize("seed,n,p,k", [(0, 30, 60, 6), (1, 30, 60, 6), (2, 40, 120, 8), (3, 50, 40, 5),
                                        (4, 20, 200, 4), (5, 64, 64, 10)])
def test_oracle_matches_the_exact_homotopy_path(seed, n, p, k):
    """The homotopy (LARS-Lasso) path gives the minimiser of eq. 2 without iterating:
    it satisfies the optimality conditions of Sec. 1 to rounding (c = K^T (y - K x)
    equals lam sgn x on the support, |c| <= lam off it, ||x||_1 = rho), and the
    oracle's Alg. GP + SS solution agrees with it: the same support and signs, x to
    1e-6, f and lam to 1e-8 (the oracle, after tens of thousands of iterations at its
    floor, sits within about 1e-11 relative of the ball's surface)."""
    rng = np.random.default_rng(seed)
    K = rng.standard_normal((n, p)) / np.sqrt(n)
    xt = np.zeros(p)
    xt[rng.choice(p, k, replace=False)] = rng.standard_normal(k)
    y = K @ xt + 0.01 * rng.standard_normal(n)
    rho = 0.8 * np.abs(xt).sum()
    xh, lam, segs = homotopy.solve_at_radius(K, y, rho)
    assert segs >= 1
    c = K.T @ (y - K @ xh)
    on = xh != 0
    assert abs(np.abs(xh).sum() - rho) <= 1e-12 * rho
    assert np.max(np.abs(c[on] - lam * np.sign(xh[on]))) <= 1e-12 * lam
    assert np.max(np.abs(c[~on])) <= lam * (1 + 1e-12)
    prob = W.Problem(np.ascontiguousarray(K), n, p, p, W.DT_F64, y, rho, xt, "homotopy")
    xo, ro, _ = oracle.reference_solve(prob)
    assert np.array_equal(np.sign(xh), np.sign(np.where(np.abs(xo) > 1e-9 * np.abs(xo).max(), xo, 0.0)))
    assert np.linalg.norm(xo - xh) <= 1e-6 * np.linalg.norm(xh)
    fh = float(np.sum((K @ xh - y) ** 2))
    assert abs(ro.f - fh) <= 1e-8 * fh
    assert abs(ro.lambda_reg - lam) <= 1e-6 * lam


def test_homotopy_path_is_piecewise_linear_and_monotone():
    """Along the path ||x(lam)||_1 grows as lam falls, and between two radii on one
    segment (same support and signs) the solution is the linear interpolation."""
    rng = np.random.default_rng(11)
    n, p = 30, 80
    K = rng.standard_normal((n, p)) / np.sqrt(n)
    xt = np.zeros(p)
    xt[rng.choice(p, 7, replace=False)] = rng.standard_normal(7)
    y = K @ xt + 0.01 * rng.standard_normal(n)
    radii = np.linspace(0.05, 0.9, 40) * np.abs(xt).sum()
    sols = [homotopy.solve_at_radius(K, y, r) for r in radii]
    lams = np.array([s[1] for s in sols])
    assert np.all(np.diff(lams) < 0)
    for (x0, _, _), (x1, _, _), (x2, _, _), r0, r1, r2 in zip(sols, sols[1:], sols[2:], radii, radii[1:], radii[2:]):
        if np.array_equal(np.sign(x0), np.sign(x1)) and np.array_equal(np.sign(x1), np.sign(x2)):
            t = (r1 - r0) / (r2 - r0)
            assert np.linalg.norm(x1 - ((1 - t) * x0 + t * x2)) <= 1e-10 * np.linalg.norm(x1)


# ------------------------------------------------------- comparison methods (Sec. 2)


def _homotopy_stored(case):
    z = np.load(os.path.join(os.path.dirname(__file__), "golden", "homotopy_small.npz"))
    return z[f"y{case}"], z[f"x{case}"], float(z[f"lam{case}"][0]), float(z[f"rho{case}"][0])


def test_ista_fista_one_step_on_orthonormal_k_is_the_closed_form():
    """K^T K = I: eq. 1 separates into p scalar problems x_i^2 - 2 x_i b_i +
    2 lam |x_i| (b = K^T y), minimised by the soft threshold S_lam(b_i).  From any
    x0 one ISTA or FISTA step (s = 1) lands there and stays: K^T K x0 = x0
    cancels the starting point, and T is constant on such a K."""
    prob = W.orthonormal(200, 80, 10, seed=4)
    K = prob.K_f64()
    b = K.T @ prob.y
    lam = 0.3 * np.abs(b).max()
    xs = np.sign(b) * np.maximum(np.abs(b) - lam, 0.0)
    # the scalar problems' minimiser, checked against a fine grid for a few entries
    for i in np.argsort(-np.abs(b))[:3]:
        grid = np.linspace(-2 * abs(b[i]), 2 * abs(b[i]), 40001)
        obj = grid ** 2 - 2 * grid * b[i] + 2 * lam * np.abs(grid)
        assert abs(grid[np.argmin(obj)] - xs[i]) <= 4 * abs(b[i]) / 40000
    x0 = np.random.default_rng(5).standard_normal(80)
    for fista in (False, True):
        for iters in (1, 3):
            x, tr = methods.ista(K, prob.y, lam, iters, step=1.0, x0=x0, fista=fista)
            np.testing.assert_allclose(x, xs, atol=1e-12 * np.abs(b).max())
    assert np.count_nonzero(xs) > 0


def test_fista_first_step_equals_ista_and_momentum_follows_t():
    """t^(0) = 1 gives no momentum in the first step, so FISTA's x^(1) is ISTA's;
    the second step's extrapolation weight is (t^(1) - 1)/t^(2) with
    t^(1) = (1 + sqrt 5)/2 and t^(2) = (1 + sqrt(1 + 4 t1^2))/2."""
    rng = np.random.default_rng(6)
    K = rng.standard_normal((20, 50)) / np.sqrt(20) / 3.0
    y = rng.standard_normal(20)
    lam = 0.05
    xi, _ = methods.ista(K, y, lam, 1)
    xf, _ = methods.ista(K, y, lam, 1, fista=True)
    assert np.array_equal(xi, xf)
    t1 = (1 + np.sqrt(5.0)) / 2
    t2 = (1 + np.sqrt(1 + 4 * t1 * t1)) / 2
    u = xf + (t1 - 1) / t2 * (xf - 0.0)
    x2 = methods.soft(u + K.T @ (y - K @ u), lam)
    np.testing.assert_allclose(methods.ista(K, y, lam, 2, fista=True)[0], x2, rtol=0, atol=1e-15)


def test_psd_hand_derived_step_on_a_diagonal_k():
    """K = diag(1, 2), y = (1, 1), x0 = 0: r = K^T y = (1, 2), ||r||^2 = 5,
    K r = (1, 4), ||K r||^2 = 17, beta = 5/17, x0 + beta r = (5/17, 10/17).
    rho = 10: inside the ball, x1 = (5/17, 10/17).  rho = 1/2: the projection
    subtracts tau = (15/17 - 1/2)/2 = 13/68 from both, x1 = (7/68, 27/68)."""
    K = np.diag([1.0, 2.0])
    y = np.array([1.0, 1.0])
    x, tr = methods.psd(K, y, 10.0, 1)
    assert abs(tr[0, 2] - 5 / 17) <= 1e-15 and abs(tr[0, 0] - 2.0) <= 1e-15
    np.testing.assert_allclose(x, [5 / 17, 10 / 17], rtol=0, atol=1e-15)
    x, _ = methods.psd(K, y, 0.5, 1)
    np.testing.assert_allclose(x, [7 / 68, 27 / 68], rtol=0, atol=1e-15)


def test_psd_one_step_on_orthonormal_k_is_the_closed_form():
    """K^T K = I: ||K r|| = ||r||, so beta = 1 and x1 = P(x0 + K^T y - x0) =
    P(K^T y), the minimiser of eq. 2 (threshold by bisection, not the oracle's
    projection)."""
    prob = W.orthonormal(300, 120, 15, seed=3, rho_scale=0.5)
    K = prob.K_f64()
    xs, tau = soft_threshold_bisect(K.T @ prob.y, prob.rho)
    x, tr = methods.psd(K, prob.y, prob.rho, 1)
    assert abs(tr[0, 2] - 1.0) <= 1e-12
    np.testing.assert_allclose(x, xs, atol=1e-12 * np.abs(xs).max())


@pytest.mark.parametrize("case", [0, 2, 4])
def test_methods_reach_the_exact_homotopy_points(case):
    """On the stored homotopy problems: ISTA and FISTA (step 1/||K||^2) reach
    x-bar(lam), the minimiser of eq. 1 at the stored lam; PSD reaches the
    minimiser of eq. 2 at the stored radius, which is the same point (the
    relation of Sec. 1)."""
    from make_golden import HOMOTOPY_CASES
    seed, n, p, k = HOMOTOPY_CASES[case]
    K, _, _, _ = W.homotopy_case(seed, n, p, k)
    y, xh, lam, rho = _homotopy_stored(case)
    s = 1.0 / np.linalg.norm(K, 2) ** 2
    xf, trf = methods.ista(K, y, lam, 20000, step=s, fista=True)
    xi, tri = methods.ista(K, y, lam, 60000, step=s)
    xp, trp = methods.psd(K, y, rho, 20000)
    for x in (xf, xi, xp):
        assert np.linalg.norm(x - xh) <= 1e-7 * np.linalg.norm(xh), np.linalg.norm(x - xh) / np.linalg.norm(xh)
    F = methods.penalised(K, y, lam, xh)
    assert trf[-1, 1] <= F * (1 + 1e-12) and tri[-1, 1] <= F * (1 + 1e-12)
    assert np.all(np.diff(tri[:, 1]) <= 1e-12 * F)      # ISTA decreases eq. 1 monotonically
