"""gpl1_solve_noalloc (the library's allocation-free solve, which keeps its
workspace in a static device array) against gpl1_solve (context workspace) on
the same instances, two calls in a row, plus its size limit.  Collected last
so that it also runs after every other GPU test in the same process."""
import numpy as np
import pytest
import torch

import oracle
import paper_0902_4424_gb300 as pkg
import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def to_dev(prob):
    K = torch.from_numpy(prob.K.view(np.int16) if prob.dtype == W.DT_BF16 else prob.K).to(DEV)
    return K, torch.from_numpy(prob.y).to(DEV)


@pytest.mark.parametrize("which", ["f32", "c0_f64", "bf16"])
def test_noalloc_matches_context_solve(gpu_ctx, which):
    if which == "f32":
        prob = W.gaussian(300, 1000, 15, dtype=W.DT_F32, seed=2101, law="gauss", sigma=0.01, rho_scale=0.8)
    elif which == "bf16":
        prob = W.gaussian(240, 960, 12, dtype=W.DT_BF16, seed=2102, law="pm1", sigma=0.01, rho_scale=1.0)
    else:
        prob = W.config0()
    fstar = oracle.reference_solve(prob)[1].f
    K, y = to_dev(prob)
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, f_star=fstar, max_iter=20000)
    x_ref, r_ref = gpu_ctx.solve(K, y, prob.rho, p=prob.p, params=prm)
    torch.cuda.synchronize()
    assert r_ref.status == 0, r_ref.as_dict()
    xr = x_ref.double().cpu().numpy()
    # x preallocated (x0 = 0 through the parameter), so that neither the C call
    # nor the wrapper allocates device memory during the calls below
    prm0 = pkg.Params.from_buffer_copy(prm)
    prm0.x0_is_zero = 1
    x = torch.full((prob.p,), float("nan"), dtype=x_ref.dtype, device=DEV)
    for call in range(2):   # the second call reuses the static scratch
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        x, r = pkg.solve_noalloc(K, y, prob.rho, x=x, p=prob.p, params=prm0)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        # the entry point's defining property: it allocates nothing.  The first
        # call may load the module that holds the static array (lazy module
        # loading), which places the array; from the second call on, free
        # device memory must not move.
        if call > 0:
            assert free_after == free_before, (call, free_before, free_after)
        assert r.status == 0 and r.stop == 0, (call, r.as_dict())
        xn = x.double().cpu().numpy()
        gap = (oracle.objective(prob, xn) - fstar) / fstar
        assert gap <= 1e-6, (call, gap)
        # both runs stop within the same 5e-7 band around f*; on these
        # well-conditioned instances that pins x to 1e-3 relative
        assert np.linalg.norm(xn - xr) <= 1e-3 * np.linalg.norm(xr), call
        assert abs(r.iters - r_ref.iters) <= max(3, r_ref.iters // 10), (r.iters, r_ref.iters)


def test_noalloc_rejects_problems_beyond_its_scratch(gpu_ctx):
    n, p = 200_000, 16       # K products need ~32 n bytes > 4 MiB
    K = torch.zeros(n, p, dtype=torch.float32, device=DEV)
    y = torch.zeros(n, dtype=torch.float32, device=DEV)
    with pytest.raises(pkg.Gpl1Error) as e:
        pkg.solve_noalloc(K, y, 1.0)
    assert e.value.status == 7 and "GPL1_NOALLOC_SCRATCH_BYTES" in str(e.value)
