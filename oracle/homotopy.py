"""Exact solution path of eq. 2 by the homotopy (LARS-Lasso) method: a second,
non-iterative reference for small problems.

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` may import this module.  It shares
no code with the CUDA library and never imports it.

The solution x(lam) of the penalised problem min 1/2 ||K x - y||^2 + lam ||x||_1
is piecewise linear in lam (Sec. 1: the solutions of eq. 1 and eq. 2 coincide
when ||x(lam)||_1 = rho, with lam = max |K^T (y - K x)|).  Starting from
lam = max |K^T y| and x = 0, the path is followed downwards segment by
segment (Osborne, Presnell and Turlach 2000; Efron, Hastie, Johnstone and
Tibshirani 2004, the Lasso modification of LARS):

  * on a segment the active set A and the signs s_A are fixed, the
    correlations c = K^T (y - K x) satisfy c_A = lam s_A, and
    x_A moves by  gamma * delta,  delta = (K_A^T K_A)^-1 s_A, as lam drops by
    gamma;
  * the segment ends where an inactive |c_j| reaches lam (j joins A) or an
    active x_j reaches 0 (j leaves A);
  * ||x||_1 = s_A^T x_A is linear on the segment, so the point with
    ||x||_1 = rho is found exactly.

Each step is a small dense solve; the path is exact up to the rounding of those
solves (it assumes general position: one event at a time).  An index that just
joined may not leave on the next segment, nor one that just left join again
(rounding would otherwise produce a step of length ~0 the wrong way), and the
result is checked against the optimality conditions before it is returned: a
path lost to rounding raises instead of returning a wrong point.
"""
from __future__ import annotations

import numpy as np


def solve_at_radius(K, y, rho: float, max_segments: int = 10000):
    """x minimising ||K x - y||^2 subject to ||x||_1 <= rho, and lam = max|K^T (y - K x)|.
    Returns (x, lam, segments walked).  If the least-squares path ends before
    ||x||_1 reaches rho (the constraint is inactive), returns the end of the path."""
    K = np.asarray(K, np.float64)
    y = np.asarray(y, np.float64)
    n, p = K.shape
    x = np.zeros(p)
    c = K.T @ y
    lam = float(np.max(np.abs(c)))
    if lam == 0.0 or rho <= 0.0:
        return x, lam, 0
    active = [int(np.argmax(np.abs(c)))]
    just_joined, just_left = active[0], -1
    for seg in range(1, max_segments + 1):
        A = np.array(active)
        s = np.sign(c[A])
        KA = K[:, A]
        delta = np.linalg.solve(KA.T @ KA, s)
        a = K.T @ (KA @ delta)           # dc/dgamma = -a
        l1 = float(np.sum(np.abs(x)))
        dl1 = float(s @ delta)           # d||x||_1 / dgamma on this segment
        # candidate events along gamma > 0
        gamma, event = lam, ("end", -1)  # lam cannot drop below 0
        inactive = np.setdiff1d(np.arange(p), A)
        for j in inactive:
            if j == just_left:
                continue
            for sgn in (1.0, -1.0):      # c_j - gamma a_j = sgn (lam - gamma)
                den = sgn - a[j]
                if den != 0.0:
                    g = (sgn * lam - c[j]) / den
                    if 0.0 < g < gamma:
                        gamma, event = g, ("join", int(j))
        for q, j in enumerate(A):
            if delta[q] != 0.0 and j != just_joined:
                g = -x[j] / delta[q]
                if 0.0 < g < gamma:
                    gamma, event = g, ("leave", int(j))
        # does ||x||_1 reach rho on this segment?
        if dl1 > 0.0 and l1 + gamma * dl1 >= rho:
            g = (rho - l1) / dl1
            x[A] += g * delta
            return _checked(K, y, x, lam - g), lam - g, seg
        x[A] += gamma * delta
        c = c - gamma * a
        lam -= gamma
        just_joined, just_left = -1, -1
        if event[0] == "join":
            active.append(event[1])
            just_joined = event[1]
        elif event[0] == "leave":
            active.remove(event[1])
            x[event[1]] = 0.0
            just_left = event[1]
        else:   # lam reached 0: the least-squares end of the path
            return x, 0.0, seg
        if len(active) > min(n, p):
            return x, lam, seg
    raise RuntimeError("homotopy did not reach the radius")


def _checked(K, y, x, lam):
    """x if it meets the optimality conditions at lam (c = K^T (y - K x) equals
    lam sgn x on the support, |c| <= lam off it, both to 1e-9 of lam); raises otherwise."""
    c = K.T @ (y - K @ x)
    on = x != 0
    if on.any() and np.max(np.abs(c[on] - lam * np.sign(x[on]))) > 1e-9 * lam:
        raise RuntimeError("homotopy: the path was lost (support conditions)")
    if (~on).any() and np.max(np.abs(c[~on])) > lam * (1 + 1e-9):
        raise RuntimeError("homotopy: the path was lost (an inactive correlation exceeds lam)")
    return x
