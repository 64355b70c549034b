"""gpl1_gemm_bf16 (tcgen05 tensor cores) against the FP64 product of the same
bfloat16 values, element by element, with the FP32-accumulation bound
|err| <= K * 2^-23 * sum_k |a_k b_k| (plus a tiny absolute floor)."""
import numpy as np
import pytest
import torch

import paper_0902_4424_gb300 as pkg
import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def bf16(rng, shape, scale=1.0):
    bits = W.f32_to_bf16_bits((rng.standard_normal(shape) * scale).astype(np.float32))
    return bits, W.bf16_bits_to_f64(bits)


@pytest.mark.parametrize("M,Ka,N,Kd", [(128, 64, 128, 64), (200, 128, 300, 128), (130, 64, 40, 192),
                                       (1024, 2048, 512, 2048), (512, 256, 1024, 768), (77, 1024, 257, 1024)])
def test_gemm_matches_fp64_product(gpu_ctx, M, Ka, N, Kd):
    rng = np.random.default_rng(M * 7 + N + Kd)
    a_bits, a = bf16(rng, (M, Ka))
    b_bits, b = bf16(rng, (N, Kd), 0.5)
    A = torch.from_numpy(a_bits.view(np.int16)).to(DEV)
    B = torch.from_numpy(b_bits.view(np.int16)).to(DEV)
    out = gpu_ctx.gemm_bf16(A, B, scale=2.0)
    torch.cuda.synchronize()
    reps = Kd // Ka
    a_rep = np.concatenate([a] * reps, axis=1)                    # A[m, k % Ka]
    exact = 2.0 * (b @ a_rep.T)                                   # out[n, m]
    bound = Kd * 2.0 ** -23 * 2.0 * (np.abs(b) @ np.abs(a_rep).T) + 1e-30
    got = out.double().cpu().numpy()
    assert got.shape == (N, M)
    err = np.abs(got - exact)
    assert np.all(err <= bound), (err.max(), (err / bound).max())


def test_gemm_rejects_bad_shapes(gpu_ctx):
    A = torch.zeros(64, 96, dtype=torch.int16, device=DEV)
    B = torch.zeros(64, 96, dtype=torch.int16, device=DEV)
    with pytest.raises(pkg.Gpl1Error) as e:
        gpu_ctx.gemm_bf16(A, B)                  # K not a multiple of 64
    assert e.value.status == 1


@pytest.mark.parametrize("config", [0, 1, 2, 3])
@pytest.mark.parametrize("splits", [1, 3, 7])
def test_gemm_configs_and_splits_add_up(gpu_ctx, config, splits):
    """Every kernel configuration, with the contraction split into parts whose
    sum (taken in order, as the shared-K solve does) is the product: each part
    within the FP32 bound of its own k-range, the sum within the bound of the whole."""
    M, Ka, N, Kd = 300, 512, 200, 1536          # ragged M and N tiles; A wraps three times
    rng = np.random.default_rng(1000 * config + splits)
    a_bits, a = bf16(rng, (M, Ka))
    b_bits, b = bf16(rng, (N, Kd), 0.5)
    A = torch.from_numpy(a_bits.view(np.int16)).to(DEV)
    B = torch.from_numpy(b_bits.view(np.int16)).to(DEV)
    parts = gpu_ctx.gemm_bf16_ex(A, B, config, splits, scale=2.0)
    torch.cuda.synchronize()
    a_rep = np.concatenate([a] * (Kd // Ka), axis=1)
    kb = Kd // 64
    total = np.zeros((N, M))
    for z in range(splits):
        k0, k1 = 64 * (z * kb // splits), 64 * ((z + 1) * kb // splits)
        exact = 2.0 * (b[:, k0:k1] @ a_rep[:, k0:k1].T)
        bound = (k1 - k0) * 2.0 ** -23 * 2.0 * (np.abs(b[:, k0:k1]) @ np.abs(a_rep[:, k0:k1]).T) + 1e-30
        got = parts[z].double().cpu().numpy()
        assert np.all(np.abs(got - exact) <= bound), (z, (np.abs(got - exact) / bound).max())
        total += got
    exact = 2.0 * (b @ a_rep.T)
    bound = (Kd + splits) * 2.0 ** -23 * 2.0 * (np.abs(b) @ np.abs(a_rep).T) + 1e-30
    assert np.all(np.abs(total - exact) <= bound)


def test_gemm_ex_rejects_bad_config(gpu_ctx):
    A = torch.zeros(128, 128, dtype=torch.int16, device=DEV)
    B = torch.zeros(128, 128, dtype=torch.int16, device=DEV)
    for cfg, spl in [(-1, 1), (4, 1), (0, 0), (0, 3)]:          # Kd / 64 = 2 parts at most
        with pytest.raises(pkg.Gpl1Error) as e:
            gpu_ctx.gemm_bf16_ex(A, B, cfg, spl)
        assert e.value.status == 1


@pytest.mark.parametrize("M,N", [(1, 1), (1, 300), (300, 1)])
def test_gemm_degenerate_output_shapes(gpu_ctx, M, N):
    """One output row or column: a single partial tile, every other row/column masked."""
    rng = np.random.default_rng(M * 1000 + N)
    a_bits, a = bf16(rng, (M, 128))
    b_bits, b = bf16(rng, (N, 128))
    A = torch.from_numpy(a_bits.view(np.int16)).to(DEV)
    B = torch.from_numpy(b_bits.view(np.int16)).to(DEV)
    out = gpu_ctx.gemm_bf16(A, B)
    torch.cuda.synchronize()
    exact = b @ a.T
    bound = 128 * 2.0 ** -23 * (np.abs(b) @ np.abs(a).T) + 1e-30
    assert np.all(np.abs(out.double().cpu().numpy() - exact) <= bound)
