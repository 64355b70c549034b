"""Seeded synthetic inputs for the l1-constrained least-squares problem (eq. 2).

This module only draws random numbers and lays them out in memory.  It holds
none of the method's arithmetic, so both sides of every comparison (the CUDA
path and the FP64 oracle under ``oracle/``) take their inputs from here and
from nowhere else.

Problem: ``min ||K x - y||^2  subject to  ||x||_1 <= rho`` (eq. 2, Sec. 1).

The paper's own test operators (Sec. 4) are a 1848x8192 Gaussian matrix scaled
to unit norm with about 2% noise and a seismic-tomography matrix that is not
public.  The workloads below keep the structure of those tests (Gaussian
compressed-sensing operators, a sparse true signal, additive Gaussian noise, an
ill-conditioned operator with a geometric singular spectrum) at the sizes the
GPU path is measured on.

Every generator uses numpy's PCG64 stream seeded with ``SEED_BASE + index`` and
produces the data in float64 before rounding it to the stored dtype with
round-to-nearest-even.  The rounded K *defines* the problem: ``y`` is formed
from the stored (rounded) K widened back to float64.
"""
from __future__ import annotations

import dataclasses
import numpy as np

SEED_BASE = 20090900

DT_F64, DT_F32, DT_BF16 = 0, 1, 2
_ITEMSIZE = {DT_F64: 8, DT_F32: 4, DT_BF16: 2}
DTYPE_NAMES = {DT_F64: "f64", DT_F32: "f32", DT_BF16: "bf16"}


def f32_to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even); returns uint16 bit patterns."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return r.astype(np.uint16)


def bf16_bits_to_f64(b: np.ndarray) -> np.ndarray:
    """Widen bfloat16 bit patterns (uint16) exactly to float64."""
    return (b.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def padded_ld(p: int, dtype: int) -> int:
    """Row stride in elements: rows start on 16-byte boundaries."""
    per16 = 16 // _ITEMSIZE[dtype]
    return ((p + per16 - 1) // per16) * per16


@dataclasses.dataclass
class Problem:
    """One instance of eq. 2 in stored form.

    ``K`` is n x ldk row-major in the stored dtype (float64/float32 numpy array,
    or uint16 bfloat16 bit patterns); columns p..ldk-1 are zero padding.
    ``y`` is float64 for DT_F64 problems and float32 otherwise.
    """
    K: np.ndarray
    n: int
    p: int
    ldk: int
    dtype: int
    y: np.ndarray
    rho: float
    x_true: np.ndarray
    name: str = ""

    def K_f64(self) -> np.ndarray:
        """The stored K widened exactly to float64, shape (n, p)."""
        if self.dtype == DT_BF16:
            return bf16_bits_to_f64(self.K[:, : self.p])
        return np.asarray(self.K[:, : self.p], dtype=np.float64)


def _store(K64: np.ndarray, dtype: int, ldk: int) -> np.ndarray:
    n, p = K64.shape
    if dtype == DT_F64:
        out = np.zeros((n, ldk), np.float64)
        out[:, :p] = K64
    elif dtype == DT_F32:
        out = np.zeros((n, ldk), np.float32)
        out[:, :p] = K64.astype(np.float32)
    else:
        out = np.zeros((n, ldk), np.uint16)
        out[:, :p] = f32_to_bf16_bits(K64.astype(np.float32))
    return out


def _sparse_signal(rng, p: int, k: int, law: str) -> np.ndarray:
    x = np.zeros(p, np.float64)
    pos = rng.permutation(p)[:k]
    if law == "pm1":          # +-1 with a fair sign
        x[pos] = np.where(rng.random(k) < 0.5, -1.0, 1.0)
    else:                     # Bernoulli-Gaussian: N(0,1) values on the support
        x[pos] = rng.standard_normal(k)
    return x


def _finish(rng, K64, dtype, x_true, sigma, rho_scale, name, ldk=None) -> Problem:
    n, p = K64.shape
    ldk = padded_ld(p, dtype) if ldk is None else ldk
    Ks = _store(K64, dtype, ldk)
    Kw = bf16_bits_to_f64(Ks[:, :p]) if dtype == DT_BF16 else np.asarray(Ks[:, :p], np.float64)
    y64 = Kw @ x_true + sigma * rng.standard_normal(n)
    y = y64 if dtype == DT_F64 else y64.astype(np.float32)
    rho = float(rho_scale * np.abs(x_true).sum())
    return Problem(Ks, n, p, ldk, dtype, y, rho, x_true, name)


def gaussian(n: int, p: int, k: int, *, dtype: int = DT_F32, seed: int = 0,
             law: str = "pm1", sigma: float = 0.01, rho_scale: float = 1.0,
             name: str = "") -> Problem:
    """Compressed-sensing instance: K iid N(0, 1/n), k-sparse x_true, y = K x_true + N(0, sigma^2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    K64 = rng.standard_normal((n, p)) / np.sqrt(n)
    x_true = _sparse_signal(rng, p, k, law)
    return _finish(rng, K64, dtype, x_true, sigma, rho_scale, name or f"gauss{n}x{p}")


def ill_conditioned(n: int, *, smin: float = 1e-4, k: int = 200, dtype: int = DT_F32,
                    seed: int = 0, sigma: float = 1e-3, name: str = "") -> Problem:
    """Square K = Q1 diag(s) Q2^T with s geometric from 1 down to smin (stand-in for the seismic operator)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Q1, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = smin ** (np.arange(n) / (n - 1))
    K64 = (Q1 * s) @ Q2.T
    x_true = _sparse_signal(rng, n, k, "gauss")
    return _finish(rng, K64, dtype, x_true, sigma, 1.0, name or f"illcond{n}")


def orthonormal(n: int, p: int, k: int, *, seed: int = 0, sigma: float = 0.01,
                rho_scale: float = 0.5) -> Problem:
    """K with orthonormal columns (K^T K = I, n >= p), FP64: the closed-form special case of eq. 2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Q, _ = np.linalg.qr(rng.standard_normal((n, p)))
    x_true = _sparse_signal(rng, p, k, "gauss")
    return _finish(rng, Q, DT_F64, x_true, sigma, rho_scale, f"orth{n}x{p}")


# --------------------------------------------------------------------------
# The measured configurations.
# --------------------------------------------------------------------------

def config0() -> Problem:
    """Plain GP, FP64: K 256x1024 N(0,1/256), 20-sparse +-1 signal, noise 0.01, rho = ||x_true||_1."""
    return gaussian(256, 1024, 20, dtype=DT_F64, seed=SEED_BASE + 0, law="pm1",
                    sigma=0.01, rho_scale=1.0, name="c0_gauss256x1024_f64")


def config1() -> Problem:
    """Compressed sensing, FP32: K 4096x16384 N(0,1/4096), 400-sparse N(0,1), noise 0.01, rho = 0.9||x_true||_1."""
    return gaussian(4096, 16384, 400, dtype=DT_F32, seed=SEED_BASE + 1, law="gauss",
                    sigma=0.01, rho_scale=0.9, name="c1_gauss4096x16384_f32")


def config2() -> Problem:
    """Ill-conditioned, FP32: K = Q1 diag(s) Q2^T 4096x4096, s from 1 to 1e-4, 200-sparse, noise 1e-3."""
    return ill_conditioned(4096, smin=1e-4, k=200, dtype=DT_F32, seed=SEED_BASE + 2,
                           sigma=1e-3, name="c2_illcond4096_f32")


def ragged_sizes(count: int = 512, nmin: int = 128, nmax: int = 2048, seed: int = SEED_BASE + 3):
    """Row counts of the ragged batch: n uniform in [nmin, nmax], p = 4n."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = rng.integers(nmin, nmax + 1, size=count)
    return [int(v) for v in n]


def ragged_instance(i: int, n: int, *, dtype: int = DT_BF16, seed: int = SEED_BASE + 3) -> Problem:
    """Instance i of the ragged batch: K n x 4n N(0,1/n), floor(n/20) entries +-1, noise 0.01."""
    return gaussian(n, 4 * n, max(1, n // 20), dtype=dtype, seed=seed * 1000 + i, law="pm1",
                    sigma=0.01, rho_scale=1.0, name=f"c3a_{i}_{n}x{4*n}")


def shared_k(n: int = 2048, p: int = 8192, nrhs: int = 1024, k: int = 102, *,
             dtype: int = DT_BF16, seed: int = SEED_BASE + 4, sigma: float = 0.01, law: str = "pm1"):
    """One K shared by nrhs right-hand sides, each from its own k-sparse signal
    (+-1 entries, or N(0,1) entries for law="gauss").

    Returns (K stored n x ldk, ldk, Y float32 nrhs x n, rho float64 nrhs, X_true nrhs x p).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    K64 = rng.standard_normal((n, p)) / np.sqrt(n)
    ldk = padded_ld(p, dtype)
    Ks = _store(K64, dtype, ldk)
    Kw = bf16_bits_to_f64(Ks[:, :p]) if dtype == DT_BF16 else np.asarray(Ks[:, :p], np.float64)
    X = np.stack([_sparse_signal(rng, p, k, law) for _ in range(nrhs)])
    Y = (X @ Kw.T + sigma * rng.standard_normal((nrhs, n))).astype(np.float32)
    rho = np.abs(X).sum(axis=1)
    return Ks, ldk, Y, rho, X


def warm_start_data(n: int = 1024, p: int = 4096, count: int = 100_000, k: int = 50, *,
                    seed: int = SEED_BASE + 5, sigma: float = 0.01):
    """Learned-warm-start recipe: K n x p N(0, 1/n) (BF16), `count` right-hand sides
    from k-sparse Bernoulli-Gaussian signals (N(0,1) values), noise sigma,
    rho = ||x_true||_1 per sample.  Returns (K, ldk, Y, rho, X_true)."""
    return shared_k(n, p, count, k, dtype=DT_BF16, seed=seed, sigma=sigma, law="gauss")


# The learned-warm-start workload as measured: training and test samples of one
# warm_start_data draw (the test samples are its last rows).
WARM_TRAIN, WARM_TEST = 16384, 256


def warm_start_split():
    """(K, ldk, Y, rho, X_true, ntrain): the measured warm-start workload, K 1024 x 4096."""
    Ks, ldk, Y, rho, X = warm_start_data(1024, 4096, WARM_TRAIN + WARM_TEST, 50)
    return Ks, ldk, Y, rho, X, WARM_TRAIN


def warm_start_train(count: int = 65536, n: int = 1024, p: int = 4096, k: int = 50, *,
                     seed: int = SEED_BASE + 6, sigma: float = 0.01):
    """More training right-hand sides for the learned warm start, on the K of
    warm_start_data (its first draw), from a separate stream: k positions drawn
    with replacement per sample (a repeated position adds its N(0,1) values),
    noise sigma, rho = ||x_true||_1.  Built sparsely, so 10^5 samples take
    seconds.  Returns (Y float32 count x n, rho float64 count)."""
    import scipy.sparse as sp
    rng_k = np.random.Generator(np.random.PCG64(SEED_BASE + 5))
    K64 = rng_k.standard_normal((n, p)) / np.sqrt(n)
    Kw = bf16_bits_to_f64(_store(K64, DT_BF16, padded_ld(p, DT_BF16))[:, :p]).astype(np.float32)
    rng = np.random.Generator(np.random.PCG64(seed))
    Y = np.empty((count, n), np.float32)
    rho = np.empty(count, np.float64)
    chunk = 8192
    for c0 in range(0, count, chunk):
        m = min(chunk, count - c0)
        idx = rng.integers(0, p, size=(m, k))
        val = rng.standard_normal((m, k))
        X = sp.csr_matrix((val.ravel(), idx.ravel(), np.arange(0, m * k + 1, k)), shape=(m, p))
        X.sum_duplicates()
        rho[c0:c0 + m] = np.asarray(abs(X).sum(axis=1)).ravel()
        Y[c0:c0 + m] = (X.astype(np.float32) @ Kw.T) + sigma * rng.standard_normal((m, n)).astype(np.float32)
    return Y, rho


# The full learned-warm-start configuration: 10^5 training and 10^4 test
# right-hand sides on the K of warm_start_data, from separate streams.
WARM_TRAIN_FULL, WARM_TEST_FULL = 100_000, 10_000


def warm_start_test(count: int = WARM_TEST_FULL, n: int = 1024, p: int = 4096, k: int = 50, *,
                    seed: int = SEED_BASE + 8, sigma: float = 0.01):
    """Test right-hand sides of the full learned-warm-start configuration, drawn as
    warm_start_train draws its samples but from their own stream.  Returns
    (Y float32 count x n, rho float64 count)."""
    return warm_start_train(count, n, p, k, seed=seed, sigma=sigma)


def warm_start_K(n: int = 1024, p: int = 4096):
    """(K stored n x ldk BF16 bits, ldk): the K of the learned-warm-start workload."""
    Ks, ldk, _, _, _ = warm_start_data(n, p, 1, 50)
    return Ks, ldk


def lista_exact_case(seed: int = 3, n: int = 64, p: int = 128, B: int = 64, L: int = 2):
    """Learned-warm-start data on which BF16 operands and FP32 sums lose nothing:
    K with one +-1 per column, W_l with one entry in {+-1, +-1/2} per row, y
    integers in [-3, 3] (half of them zero), thresholds 3/4, targets multiples of
    1/4.  Every value the network and its gradient form is then a short dyadic
    fraction, so a BF16/FP32 implementation must return the FP64 values exactly
    (the default seed is one for which that holds).  Returns (K, W, theta, Y, Xt)
    in float64."""
    rng = np.random.default_rng(seed)
    K = np.zeros((n, p))
    rows = rng.integers(0, n, size=p)
    K[rows, np.arange(p)] = rng.choice([-1.0, 1.0], size=p)
    W = np.zeros((L, p, n))
    for l in range(L):
        for i in range(p):
            col = rng.integers(0, n)
            W[l, i, col] = rng.choice([-1.0, 1.0, 0.5, -0.5])
    Y = rng.integers(-3, 4, size=(B, n)).astype(np.float64) * (rng.random((B, n)) < 0.5)
    theta = np.full(L, 0.75)
    Xt = rng.integers(-2, 3, size=(B, p)).astype(np.float64) * 0.25 * (rng.random((B, p)) < 0.3)
    return K, W, theta, Y, Xt


def homotopy_case(seed: int, n: int, p: int, k: int):
    """A small FP64 problem for the exact homotopy reference: K n x p N(0, 1/n),
    k-sparse N(0,1) signal, noise 0.01, rho = 0.8 ||x_true||_1.  Returns
    (K, y, rho, x_true)."""
    rng = np.random.default_rng(seed)
    K = rng.standard_normal((n, p)) / np.sqrt(n)
    xt = np.zeros(p)
    xt[rng.choice(p, k, replace=False)] = rng.standard_normal(k)
    y = K @ xt + 0.01 * rng.standard_normal(n)
    return K, y, 0.8 * float(np.abs(xt).sum()), xt


def rho_sweep(n: int = 1848, p: int = 8192, k: int = 120, count: int = 50, *, seed: int = SEED_BASE + 7,
              noise: float = 0.02, lo: float = 0.05, hi: float = 1.0):
    """The paper's Gaussian test shape (Sec. 4) as a sweep over the radius: K
    n x p N(0,1) scaled to ||K||_2 = 1 (power iteration on the float64 draw),
    stored BF16 with its rows padded with zeros to a multiple of 64 (zero rows
    leave eq. 2 unchanged); x_true k-sparse N(0,1); y = K x_true + e with
    ||e|| = noise ||K x_true||; `count` radii geometric from lo to hi times
    ||x_true||_1.  Returns (K stored n_pad x ldk, ldk, n_pad, y float32 n_pad,
    rho float64 count, x_true)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    G = rng.standard_normal((n, p))
    v = rng.standard_normal(p)
    for _ in range(60):   # power iteration for ||G||_2
        w = G.T @ (G @ v)
        v = w / np.linalg.norm(w)
    K64 = G / np.sqrt(np.linalg.norm(G.T @ (G @ v)))
    n_pad = ((n + 63) // 64) * 64
    Kp = np.zeros((n_pad, p))
    Kp[:n] = K64
    ldk = padded_ld(p, DT_BF16)
    Ks = _store(Kp, DT_BF16, ldk)
    Kw = bf16_bits_to_f64(Ks[:, :p])
    x_true = _sparse_signal(rng, p, k, "gauss")
    clean = Kw @ x_true
    e = rng.standard_normal(n_pad)
    e[n:] = 0.0
    y = (clean + noise * np.linalg.norm(clean) / np.linalg.norm(e) * e).astype(np.float32)
    rho = np.abs(x_true).sum() * np.geomspace(lo, hi, count)
    return Ks, ldk, n_pad, y, rho, x_true
