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
    return solve_at_radii(K, y, [rho], max_segments)[0]


def solve_at_radii(K, y, radii, max_segments: int = 10000):
    """solve_at_radius for several radii in one walk down the path: a list of
    (x, lam, segments walked) in the order of `radii`.  The walk is the same for
    every radius, so each entry equals the single-radius result."""
    K = np.asarray(K, np.float64)
    y = np.asarray(y, np.float64)
    n, p = K.shape
    order = np.argsort(np.asarray(radii, np.float64), kind="stable")
    out = [None] * len(order)
    pending = [int(i) for i in order]          # radii not reached yet, smallest first
    x = np.zeros(p)
    c = K.T @ y
    lam = float(np.max(np.abs(c)))
    for i in list(pending):
        if lam == 0.0 or radii[i] <= 0.0:
            out[i] = (x.copy(), lam, 0)
            pending.remove(i)
    if not pending:
        return out
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
        # the first event along gamma in (0, lam): an inactive correlation
        # reaching +-(lam - gamma) (the smallest index, + before -, on ties), else
        # an active entry reaching 0 strictly earlier
        gamma, event = lam, ("end", -1)
        inactive = np.setdiff1d(np.arange(p), A)
        if just_left >= 0:
            inactive = inactive[inactive != just_left]
        if inactive.size:
            sg = np.array([1.0, -1.0])
            den = sg[None, :] - a[inactive][:, None]
            with np.errstate(divide="ignore", invalid="ignore"):
                g = (sg[None, :] * lam - c[inactive][:, None]) / den
            g = np.where((den != 0.0) & (g > 0.0) & (g < gamma), g, np.inf).ravel()
            q = int(np.argmin(g))
            if np.isfinite(g[q]):
                gamma, event = float(g[q]), ("join", int(inactive[q // 2]))
        with np.errstate(divide="ignore", invalid="ignore"):
            gl = -x[A] / delta
        gl = np.where((delta != 0.0) & (A != just_joined) & (gl > 0.0) & (gl < gamma), gl, np.inf)
        if gl.size:
            q = int(np.argmin(gl))
            if np.isfinite(gl[q]):
                gamma, event = float(gl[q]), ("leave", int(A[q]))
        # the radii that ||x||_1 reaches on this segment
        while pending and dl1 > 0.0 and l1 + gamma * dl1 >= radii[pending[0]]:
            i = pending.pop(0)
            g = (radii[i] - l1) / dl1
            xr = x.copy()
            xr[A] += g * delta
            out[i] = (_checked(K, y, xr, lam - g), lam - g, seg)
        if not pending:
            return out
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
        if event[0] == "end" or len(active) > min(n, p):
            # the least-squares end of the path (lam = 0) or a full active set:
            # the constraint is inactive for the radii left
            for i in pending:
                out[i] = (x.copy(), 0.0 if event[0] == "end" else lam, seg)
            return out
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
