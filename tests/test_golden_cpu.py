"""The stored minimisers in tests/golden/ against what fixes them independently
of the run that wrote them: the optimality conditions of Sec. 1 (with
c = K^T (y - K x) and lam = max|c|: c_i = lam sgn x_i on the support,
|c_i| <= lam off it, ||x||_1 = rho), the stored optimal values, a fresh walk of
the homotopy path, and the agreement of the two oracles (Alg. GP + SS run to its
floor, and the homotopy path) on the radius sweep."""
import json
import os
import sys

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import homotopy

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
from make_golden import HOMOTOPY_CASES, load_sparse  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def conditions(prob, x):
    """(f, support residual / lam, max off-support |c| / lam, | ||x||_1 - rho | / rho)."""
    f, lam, fw, g = oracle.certificates(prob, x)
    c = -0.5 * g
    on = x != 0
    return (f, float(np.abs(c[on] - lam * np.sign(x[on])).max() / lam),
            float(np.abs(c[~on]).max() / lam), abs(float(np.abs(x).sum()) - prob.rho) / prob.rho)


def check(prob, x, f_star, supp_bar, f_bar=1e-12):
    f, supp, off, l1 = conditions(prob, x)
    assert abs(f - f_star) <= f_bar * f_star, (prob.name, f, f_star)
    assert supp <= supp_bar, (prob.name, supp)
    assert off <= 1.0 + 1e-9, (prob.name, off)
    assert l1 <= 1e-12, (prob.name, l1)


@pytest.mark.parametrize("name", ["c0", "c1", "c2"])
def test_stored_xstar_of_the_configs(name):
    prob = {"c0": W.config0, "c1": W.config1, "c2": W.config2}[name]()
    xs, meta = load_sparse(os.path.join(GOLD, f"xstar_{name}.npz"))
    f_star = json.load(open(os.path.join(GOLD, "fstar.json")))[name]["f_star"]
    assert meta["f"] == f_star
    check(prob, xs[0], f_star, supp_bar=1e-5)


def test_stored_xstar_of_the_ragged_batch_sample():
    xs, meta = load_sparse(os.path.join(GOLD, "xstar_c3a.npz"))
    fs = json.load(open(os.path.join(GOLD, "c3a_fstar.json")))["f_star"]
    sizes = W.ragged_sizes(512)
    assert len(xs) == 16
    for i, x in zip(meta["instances"], xs):
        check(W.ragged_instance(i, sizes[i]), x, fs[i], supp_bar=1e-5)


def test_stored_xstar_of_the_shared_k_and_warm_start_samples():
    xs, meta = load_sparse(os.path.join(GOLD, "xstar_c3b.npz"))
    fs = json.load(open(os.path.join(GOLD, "c3b_fstar.json")))["f_star"]
    Ks, ldk, Y, rho, X = W.shared_k(nrhs=1024)
    n, p = Ks.shape[0], X.shape[1]
    for b, x in zip(meta["instances"], xs):
        check(W.Problem(Ks, n, p, ldk, W.DT_BF16, Y[b].copy(), float(rho[b]), X[b], f"c3b_{b}"), x, fs[b], 1e-5)
    xs, meta = load_sparse(os.path.join(GOLD, "xstar_c4.npz"))
    fs = json.load(open(os.path.join(GOLD, "c4_fstar.json")))["f_star"]
    Ks, ldk, Y, rho, X, ntr = W.warm_start_split()
    n, p = Ks.shape[0], X.shape[1]
    for q, x in zip(meta["test_samples"], xs):
        b = ntr + q
        check(W.Problem(Ks, n, p, ldk, W.DT_BF16, Y[b].copy(), float(rho[b]), X[b], f"c4_{q}"), x, fs[q], 1e-5)


def test_radius_sweep_homotopy_points_and_oracle_agree():
    """Every radius: the homotopy point meets the conditions to rounding and has
    the oracle's optimal value; at every 5th radius the oracle's x* is within
    1e-6 of it (two methods that share nothing but the problem)."""
    xbar, hmeta = load_sparse(os.path.join(GOLD, "xbar_c5.npz"))
    xs, meta = load_sparse(os.path.join(GOLD, "xstar_c5.npz"))
    fs = json.load(open(os.path.join(GOLD, "c5_fstar.json")))["f_star"]
    Ks, ldk, n, y, rho, xt = W.rho_sweep()
    p = xt.shape[0]
    assert len(xbar) == len(rho)
    for b in range(len(rho)):
        prob = W.Problem(Ks, n, p, ldk, W.DT_BF16, y.copy(), float(rho[b]), xt, f"c5_{b}")
        check(prob, xbar[b], fs[b], supp_bar=1e-10, f_bar=1e-11)
    for b, x in zip(meta["radii"], xs):
        assert np.linalg.norm(x - xbar[b]) <= 1e-6 * np.linalg.norm(xbar[b]), b
        assert np.array_equal(np.sign(x), np.sign(xbar[b])), b


@pytest.mark.parametrize("case", range(len(HOMOTOPY_CASES)))
def test_stored_homotopy_points_equal_a_fresh_walk(case):
    seed, n, p, k = HOMOTOPY_CASES[case]
    K, y, rho, _ = W.homotopy_case(seed, n, p, k)
    z = np.load(os.path.join(GOLD, "homotopy_small.npz"))
    np.testing.assert_allclose(z[f"y{case}"], y, rtol=1e-14, atol=1e-15)
    assert float(z[f"rho{case}"][0]) == rho
    xh, lam, _ = homotopy.solve_at_radius(K, z[f"y{case}"], rho)
    np.testing.assert_allclose(z[f"x{case}"], xh, rtol=0, atol=1e-12 * np.abs(xh).max())
    assert abs(float(z[f"lam{case}"][0]) - lam) <= 1e-12 * lam


def test_homotopy_walk_at_several_radii_equals_single_walks():
    """solve_at_radii (one walk, radii in any order) returns what solve_at_radius
    returns for each radius alone."""
    K, y, rho, _ = W.homotopy_case(2, 40, 120, 8)
    radii = [rho, 0.3 * rho, 0.05 * rho, 0.7 * rho]
    many = homotopy.solve_at_radii(K, y, radii)
    for r, (x, lam, seg) in zip(radii, many):
        x1, lam1, seg1 = homotopy.solve_at_radius(K, y, r)
        assert np.array_equal(x, x1) and lam == lam1 and seg == seg1


def test_stored_optima_of_the_full_warm_start_test_set():
    """tests/golden/c4full_fstar.json (10^4 warm-start test samples): three entries
    recomputed by the oracle's floor solve, and every value positive and finite."""
    gold = json.load(open(os.path.join(GOLD, "c4full_fstar.json")))
    fs = gold["f_star"]
    assert len(fs) == W.WARM_TEST_FULL and all(np.isfinite(fs)) and min(fs) > 0
    Ks, ldk = W.warm_start_K()
    Y, rho = W.warm_start_test()
    for q in (0, 5000, W.WARM_TEST_FULL - 1):
        prob = W.Problem(Ks, Ks.shape[0], 4096, ldk, W.DT_BF16, Y[q].copy(), float(rho[q]), None, f"c4f_{q}")
        f = oracle.floor_solve(prob)[1].f
        assert abs(f - fs[q]) <= 1e-12 * fs[q], (q, f, fs[q])
