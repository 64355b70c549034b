"""FP64 oracle of the learned warm start: an unrolled, learned version of the
ISTA iteration of Sec. 2 (soft-thresholded Landweber steps on eq. 1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs may import this module.  It shares no code with the
CUDA library and never imports it.

Network (L layers; per layer a p x n matrix W_l and a scalar threshold theta_l):

    x^0 = 0,   z^l = x^l + W_l (y - K x^l),   x^{l+1} = S_{theta_l}(z^l),

S_t the soft threshold sgn(z) max(|z| - t, 0).  With W_l = K^T and theta_l =
lambda every layer is one ISTA step for eq. 1 (||K|| <= 1); with W_l = K^T / L,
theta_l = lambda / L (L = ||K||_2^2) one ISTA step of the rescaled problem.  The
warm start for Alg. GP is the projection of x^L onto the l1 ball of eq. 2.

Training loss over a batch of B samples with targets xt (solutions of eq. 2):
    loss = (1/B) sum_b ||x^L_b - xt_b||^2.
Backward (one subgradient of S: dS/dz = 1[|z| > t], dS/dt = -sgn(z) 1[|z| > t]):
    g^L     = (2/B)(x^L - xt)
    delta_l = g^{l+1} * 1[|z^l| > theta_l]
    dtheta_l = -sum delta_l * sgn(z^l)
    dW_l    = sum_b delta_l,b (y_b - K x^l_b)^T
    g^l     = delta_l - K^T W_l^T delta_l

Pins (tests/test_oracle_pins.py): one layer on an orthonormal K is the closed-
form minimiser of eq. 1; many tied ISTA layers reach the optimality conditions
of eq. 1 (|K^T (y - Kx)| <= lambda, equality with the sign of x on the
support); the backward pass against central finite differences.  The BF16
precision model (rounded=True): the rounding against torch's bfloat16
conversion; with data whose products need no rounding it equals the FP64
network; and its distance to the FP64 network stays within the BF16 error
bound.
"""
from __future__ import annotations

import numpy as np


def soft(z, t):
    return np.sign(z) * np.maximum(np.abs(z) - t, 0.0)


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64: the 16
    high bits of the float32 pattern after adding half of the dropped part
    (0x7fff, plus 1 when the kept part is odd).  Finite inputs only."""
    b = np.ascontiguousarray(np.asarray(a, np.float32)).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _precision(rounded: bool):
    """(operand rounding of a product, rounding of a stored value): identity in
    FP64, or BF16 operands and FP32 values (the tensor-core precision model)."""
    if not rounded:
        ident = lambda a: np.asarray(a, np.float64)   # noqa: E731
        return ident, ident
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)   # noqa: E731
    return bf16, f32


def forward(K, W, theta, Y, rounded: bool = False):
    """K (n, p); W (L, p, n); theta (L,); Y (B, n).  Returns (xs, zs): xs[l] (B, p)
    for l = 0..L (xs[0] = 0) and zs[l] (B, p) the pre-threshold values of layer l.

    rounded=True is the precision model of a tensor-core implementation: the
    operands of every matrix product rounded to BF16 (products summed exactly
    here, in FP32 there), every stored result and elementwise step in FP32."""
    op, st = _precision(rounded)
    K = np.asarray(K, np.float64)
    Y = st(Y)
    L = W.shape[0]
    B, p = Y.shape[0], K.shape[1]
    xs = [np.zeros((B, p))]
    zs = []
    for l in range(L):
        r = st(Y - st(op(xs[l]) @ op(K).T))                 # y - K x^l, per sample
        z = st(xs[l] + st(op(r) @ op(W[l]).T))
        zs.append(z)
        xs.append(st(soft(z, st(theta[l]))))
    return xs, zs


def loss(xL, Xt):
    d = xL - np.asarray(Xt, np.float64)
    return float(np.sum(d * d) / d.shape[0])


def backward(K, W, theta, Y, Xt, rounded: bool = False):
    """Loss and its gradients (dW (L, p, n), dtheta (L,)) for one batch
    (rounded: the precision model of forward)."""
    op, st = _precision(rounded)
    K = np.asarray(K, np.float64)
    xs, zs = forward(K, W, theta, Y, rounded)
    Y = st(Y)
    L = W.shape[0]
    B = Y.shape[0]
    g = st(2.0 / B * st(xs[L] - st(Xt)))
    dW = np.zeros(W.shape)
    dtheta = np.zeros(L)
    for l in range(L - 1, -1, -1):
        act = np.abs(zs[l]) > st(theta[l])
        delta = g * act
        dtheta[l] = -np.sum(delta * np.sign(zs[l]))
        r = st(Y - st(op(xs[l]) @ op(K).T))
        dW[l] = st(op(delta).T @ op(r))
        g = st(delta - st(op(st(op(delta) @ op(W[l]))) @ op(K)))
    return loss(xs[L], Xt), dW, dtheta


def spectral_norm_sq(K, iters: int = 200, seed: int = 0) -> float:
    """||K||_2^2 by power iteration on K^T K."""
    K = np.asarray(K, np.float64)
    v = np.random.default_rng(seed).standard_normal(K.shape[1])
    v /= np.linalg.norm(v)
    s = 0.0
    for _ in range(iters):
        w = K.T @ (K @ v)
        s = float(np.linalg.norm(w))
        v = w / s
    return s


def init_params(K, layers: int, lam: float):
    """W_l = K^T / L and theta_l = lam / L with L = ||K||_2^2 (ISTA's step)."""
    Lk = spectral_norm_sq(K)
    W = np.repeat((np.asarray(K, np.float64).T / Lk)[None], layers, axis=0)
    return W, np.full(layers, lam / Lk), Lk


def project_l1(x, rho):
    """Projection of one vector onto {||w||_1 <= rho} (the main oracle's
    sort-based projection), giving the warm start x0 = P(x^L)."""
    from . import project
    return project(np.asarray(x, np.float64), rho)[0]
