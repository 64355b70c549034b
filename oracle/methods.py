"""FP64 oracle of the comparison methods of Sec. 2: ISTA, FISTA (eq. fista) and
projected steepest descent (PSD), written out step by step as the paper states
them.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs may import this module.  It shares no code with the
CUDA library and never imports it.

ISTA and FISTA minimise eq. 1, ||K x - y||^2 + 2 lam ||x||_1:

    ISTA:   x^(k+1) = S_lam[x^(k) + r^(k)],   r^(k) = K^T (y - K x^(k)),
    FISTA:  x^(k+1) = T(x^(k) + (t^(k) - 1)/t^(k+1) (x^(k) - x^(k-1))),
            T(x) = S_lam[x + K^T (y - K x)],  t^(k+1) = (1 + sqrt(1 + 4 t^(k)^2))/2,
            t^(0) = 1 (so the first step carries no momentum),

with S_lam the componentwise soft threshold.  The paper states both for
||K|| < 1 (ISTA converges for ||K|| < sqrt(2)).  For a general K both take a
step s: the same iteration on the rescaled problem sqrt(s) K, sqrt(s) y,
s lam, i.e. x + s K^T (y - K x) thresholded at s lam; s = 1 is the paper's
iteration, s = 1/||K||^2 makes any K admissible.

PSD minimises eq. 2 over the l1 ball Omega of radius rho:

    x^(k+1) = P_Omega[x^(k) + beta^(k) r^(k)],   beta^(k) = ||r^(k)||^2 / ||K r^(k)||^2.

Each function returns the final iterate and a trace with one row per
iteration k (the values at x^(k), before the step): the data misfit
||K x^(k) - y||^2, the objective of the method's problem (eq. 1 for ISTA and
FISTA, eq. 2 for PSD), and the step taken (s for ISTA/FISTA, beta for PSD).

Pins (tests/test_oracle_pins.py): on an orthonormal K one step of each is the
closed-form minimiser (S_lam(K^T y) for eq. 1, P(K^T y) for eq. 2); a
hand-derived PSD step on a diagonal K; FISTA's t sequence and its first step
equal to ISTA's; all three reach the exact minimiser of the homotopy path
(eq. 1 at its lambda, eq. 2 at its radius).
"""
from __future__ import annotations

import numpy as np


def soft(v, t):
    """S_t: sgn(v) max(|v| - t, 0), componentwise."""
    return np.sign(v) * np.maximum(np.abs(v) - t, 0.0)


def penalised(K, y, lam, x):
    """The objective of eq. 1: ||K x - y||^2 + 2 lam ||x||_1."""
    r = K @ x - y
    return float(r @ r + 2.0 * lam * np.abs(x).sum())


def ista(K, y, lam: float, iters: int, step: float = 1.0, x0=None, fista: bool = False):
    """ISTA (fista=False) or FISTA (fista=True) on eq. 1 with step s = `step`.
    Returns (x^(iters), trace rows (misfit, eq. 1 objective, s))."""
    K = np.asarray(K, np.float64)
    y = np.asarray(y, np.float64)
    x = np.zeros(K.shape[1]) if x0 is None else np.array(x0, np.float64, copy=True)
    x_prev = x.copy()
    t = 1.0
    rows = []
    for _ in range(iters):
        r = K @ x - y
        rows.append((float(r @ r), float(r @ r + 2.0 * lam * np.abs(x).sum()), step))
        if fista:
            t_next = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
            u = x + (t - 1.0) / t_next * (x - x_prev)
            t = t_next
        else:
            u = x
        x_prev = x
        x = soft(u + step * (K.T @ (y - K @ u)), step * lam)
    return x, np.array(rows).reshape(-1, 3)


def psd(K, y, rho: float, iters: int, x0=None):
    """Projected steepest descent on eq. 2 from x^(0) = P_Omega(x0) (0 by
    default).  Returns (x^(iters), trace rows (misfit, misfit, beta)); stops
    early at a point where K r = 0."""
    from . import project
    K = np.asarray(K, np.float64)
    y = np.asarray(y, np.float64)
    x = np.zeros(K.shape[1]) if x0 is None else project(np.asarray(x0, np.float64), rho)[0]
    rows = []
    for _ in range(iters):
        e = y - K @ x
        r = K.T @ e
        Kr = K @ r
        den = float(Kr @ Kr)
        f = float(e @ e)
        if den == 0.0:
            break
        beta = float(r @ r) / den
        rows.append((f, f, beta))
        x = project(x + beta * r, rho)[0]
    return x, np.array(rows).reshape(-1, 3)
