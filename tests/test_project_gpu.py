"""gpl1_project (the projection P_Omega of Alg. GP, Step 2) against the FP64 oracle.

Bit-exact identity inside the ball; outside it, element-wise agreement with
the oracle's sort-based projection of the same stored values, within the
rounding of the output type (FP64: 1e-12 of max|v|; FP32: 4 ulp of max|v|,
since the GPU subtracts a float-rounded tau in float arithmetic).
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

DEV = "cuda"


def check(ctx, v, rhos):
    vt = torch.from_numpy(v).to(DEV)
    tau = torch.empty(v.shape[0], dtype=torch.float64, device=DEV)
    out = ctx.project(vt, list(rhos), tau=tau).cpu().numpy()
    tau = tau.cpu().numpy()
    for b, rho in enumerate(rhos):
        vb = v[b].astype(np.float64)
        ref, tref = oracle.project(vb, rho)
        if np.abs(vb).sum() <= rho:
            assert np.array_equal(out[b], v[b]), "identity inside the ball must be bit-exact"
            assert tau[b] == 0.0
            continue
        scale = np.abs(vb).max()
        if v.dtype == np.float64:
            np.testing.assert_allclose(out[b], ref, rtol=0, atol=1e-12 * scale)
            assert abs(tau[b] - tref) <= 1e-12 * scale
            assert abs(np.abs(out[b]).sum() - rho) <= 1e-11 * rho + 1e-12 * scale
        else:
            np.testing.assert_allclose(out[b].astype(np.float64), ref, rtol=0, atol=4 * 2.0 ** -24 * scale)
            assert abs(tau[b] - tref) <= 1e-12 * scale + 1e-15
            nz = ref != 0
            assert abs(np.abs(out[b].astype(np.float64)).sum() - rho) <= 1e-6 * rho + nz.sum() * 2.0 ** -24 * scale
        assert np.all(np.sign(out[b]) * np.sign(vb) >= 0)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("p", [1, 7, 480, 481, 1000, 4097])
def test_project_random(gpu_ctx, dtype, p):
    rng = np.random.default_rng(p)
    v = (rng.standard_normal((4, p)) * np.exp(rng.standard_normal((4, p)))).astype(dtype)
    l1 = np.abs(v.astype(np.float64)).sum(axis=1)
    rhos = [l1[0] * 0.3, l1[1] * 1e-3, l1[2] * 1.5, l1[3] * 0.97]
    check(gpu_ctx, v, rhos)


@pytest.mark.parametrize("dtype,p", [(np.float32, 16800), (np.float64, 7680), (np.float32, 16384)])
def test_project_max_size(gpu_ctx, dtype, p):
    rng = np.random.default_rng(3)
    v = rng.standard_normal((3, p)).astype(dtype)
    l1 = np.abs(v.astype(np.float64)).sum(axis=1)
    check(gpu_ctx, v, [l1[0] * 0.05, l1[1] * 0.5, 0.01])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_project_ties_zeros_tiny(gpu_ctx, dtype):
    rng = np.random.default_rng(9)
    p = 3000
    ties = rng.integers(-5, 6, size=p).astype(dtype)                       # many equal |v|, zeros
    tiny = (rng.standard_normal(p) * 1e-30).astype(dtype)                  # deep exponents
    mixed = np.where(rng.random(p) < 0.5, 0.0, rng.standard_normal(p) * 1e3).astype(dtype)
    wide = (rng.standard_normal(p) * 10.0 ** rng.uniform(-20, 20, p)).astype(dtype)
    v = np.stack([ties, tiny, mixed, wide])
    l1 = np.abs(v.astype(np.float64)).sum(axis=1)
    check(gpu_ctx, v, [l1[0] * 0.4, l1[1] * 0.2, l1[2] * 0.01, l1[3] * 0.5])


def test_project_many_segments_strided(gpu_ctx):
    rng = np.random.default_rng(21)
    batch, p, stride = 300, 777, 800
    buf = rng.standard_normal((batch, stride)).astype(np.float32)
    rhos = rng.uniform(0.1, 50, batch)
    vt = torch.from_numpy(buf).to(DEV)
    out = torch.zeros_like(vt)
    import ctypes
    import paper_0902_4424_gb300 as pkg
    rh = torch.tensor(rhos, dtype=torch.float64, device=DEV)
    st = pkg.lib().gpl1_project(gpu_ctx._h, ctypes.c_void_p(vt.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                pkg.F32, p, batch, stride, ctypes.c_void_p(rh.data_ptr()), 1, None)
    assert st == 0
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    for b in range(0, batch, 37):
        ref, _ = oracle.project(buf[b, :p].astype(np.float64), rhos[b])
        np.testing.assert_allclose(o[b, :p], ref, rtol=0, atol=4 * 2.0 ** -24 * np.abs(buf[b, :p]).max())
        assert np.all(o[b, p:] == 0)            # columns past p are not written


def test_project_in_place_and_errors(gpu_ctx):
    import paper_0902_4424_gb300 as pkg
    v = torch.randn(2, 5000, dtype=torch.float64, device=DEV)
    ref = [oracle.project(v[b].cpu().numpy(), 3.0)[0] for b in range(2)]
    gpu_ctx.project(v, 3.0, out=v)
    for b in range(2):
        np.testing.assert_allclose(v[b].cpu().numpy(), ref[b], atol=1e-12 * 5)
    with pytest.raises(pkg.Gpl1Error) as e:
        gpu_ctx.project(torch.randn(20000, device=DEV), 1.0)
    assert e.value.status == 7
    with pytest.raises(pkg.Gpl1Error) as e:
        gpu_ctx.project(torch.randn(100, device=DEV), -1.0)
    assert e.value.status == 1
