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
