"""Box shapes of the two-pass kernel (gpl1_params.tile: TMA boxes of 15, 30
or 60 KiB through the same 120 KiB ring) and the batched autotuner that picks
one per batch.  Every shape solves the same ragged batch to the FP64 oracle's
optima (relative objective gap <= 1e-6, feasibility), row counts that are not
multiples of any box height included; the tuner lists its choice and the time
of every candidate, keeps it for the context, and its choice gives the same
iterates as the shape pinned by hand; a shape the dtype has not is refused."""
import numpy as np
import pytest
import torch

import oracle
import paper_0902_4424_gb300 as pkg
import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def upload(prob):
    if prob.dtype == W.DT_BF16:
        K = torch.from_numpy(prob.K.view(np.int16)).to(DEV)
    else:
        K = torch.from_numpy(prob.K).to(DEV)
    y = torch.from_numpy(prob.y).to(DEV)
    x = torch.zeros(prob.p, dtype=torch.float64 if prob.dtype == W.DT_F64 else torch.float32, device=DEV)
    return K, y, x


def batch(dtype, count=24, seed=23):
    rng = np.random.default_rng(seed)
    sizes = [int(v) for v in rng.integers(16, 300, size=count)]
    sizes[:3] = [1, 29, 121]   # ragged against boxes of 15, 30, 60 and 120 rows
    return [W.gaussian(n, 4 * n, max(1, n // 20), dtype=dtype, seed=3000 + i, law="pm1")
            for i, n in enumerate(sizes)]


def run_batch(ctx, probs, dtype, fstars, tile):
    keep, descs = [], []
    for pr, fs in zip(probs, fstars):
        K, y, x = upload(pr)
        keep.append((K, y, x))
        descs.append(pkg.Context.make_problem(K, y, pr.rho, x, pr.p, fs))
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, x0_is_zero=1, max_iter=20000, tile=tile)
    res = ctx.solve_batched(descs, dtype, prm)
    torch.cuda.synchronize()
    return [k[2].double().cpu().numpy() for k in keep], res


def check(probs, xs, res, refs):
    for pr, x, r, fs in zip(probs, xs, res, refs):
        f = oracle.objective(pr, x)
        assert r.status == 0, (pr.n, r.as_dict(), f, fs)
        assert (f - fs) <= 1e-6 * fs + 1e-12, (pr.n, f, fs)
        assert np.abs(x).sum() <= pr.rho * (1 + 1e-6)


@pytest.mark.parametrize("dtype,tile", [
    (W.DT_BF16, pkg.TILE_SMALL), (W.DT_BF16, pkg.TILE_MEDIUM), (W.DT_BF16, pkg.TILE_LARGE),
    (W.DT_F32, pkg.TILE_SMALL), (W.DT_F32, pkg.TILE_LARGE),
    (W.DT_F64, pkg.TILE_MEDIUM), (W.DT_F64, pkg.TILE_LARGE)])
def test_every_tile_reaches_the_oracle(gpu_ctx, dtype, tile):
    probs = batch(dtype)
    refs = [oracle.reference_solve(p)[1].f for p in probs]
    xs, res = run_batch(gpu_ctx, probs, dtype, refs, tile)
    check(probs, xs, res, refs)


@pytest.mark.parametrize("tile", [pkg.TILE_SMALL, pkg.TILE_LARGE])
def test_single_two_pass_solve_with_a_pinned_tile(gpu_ctx, tile):
    """A single instance over all SMs (cooperative launch) in the small and the
    large box shape: several strips and a ragged last box of rows."""
    pr = W.gaussian(1000, 5000, 50, dtype=W.DT_F32, seed=31, law="pm1")
    fs = oracle.reference_solve(pr)[1].f
    K, y, _ = upload(pr)
    prm = pkg.params_default(stop_rule=pkg.STOP_ON_REL_GAP, tol=5e-7, f_star=fs, x0_is_zero=1, max_iter=20000,
                             engine=pkg.ENGINE_TWO_PASS, tile=tile)
    x, r = gpu_ctx.solve(K, y, pr.rho, p=pr.p, params=prm)
    xh = x.double().cpu().numpy()
    assert r.status == 0, r.as_dict()
    assert (oracle.objective(pr, xh) - fs) <= 1e-6 * fs
    assert np.abs(xh).sum() <= pr.rho * (1 + 1e-6)


def test_batched_tuner_lists_and_keeps_its_choice():
    """AUTO on a fresh context: one tuned entry keyed by (dtype, count, sum n p,
    max n p) with a time for every admissible shape; the same batch again uses
    the kept choice (no new entry); pinning the chosen shape by hand gives the
    same iterates bit for bit (the same kernel on the same instances)."""
    torch.cuda.set_device(0)
    ctx = pkg.Context(0)
    dtype = W.DT_BF16
    probs = batch(dtype, count=20, seed=29)
    refs = [oracle.reference_solve(p)[1].f for p in probs]
    xs, res = run_batch(ctx, probs, dtype, refs, pkg.TILE_AUTO)
    check(probs, xs, res, refs)
    tuned = ctx.batched_tuned()
    assert len(tuned) == 1
    t = tuned[0]
    assert t["key"] == (dtype, len(probs), sum(p.n * p.p for p in probs), max(p.n * p.p for p in probs))
    assert t["tile"] in (pkg.TILE_SMALL, pkg.TILE_MEDIUM, pkg.TILE_LARGE)
    assert all(ms > 0 for ms in t["ms"]), t
    assert t["ms"][t["tile"] - pkg.TILE_SMALL] == min(t["ms"])
    xs2, _ = run_batch(ctx, probs, dtype, refs, pkg.TILE_AUTO)
    assert len(ctx.batched_tuned()) == 1
    xs3, _ = run_batch(ctx, probs, dtype, refs, t["tile"])
    for a, b, c in zip(xs, xs2, xs3):
        assert np.array_equal(a, b) and np.array_equal(a, c)
    # FP64 has no SMALL shape: no time for it, and pinning it is refused
    p64 = batch(W.DT_F64, count=6, seed=37)
    r64 = [oracle.reference_solve(p)[1].f for p in p64]
    run_batch(ctx, p64, W.DT_F64, r64, pkg.TILE_AUTO)
    t64 = [e for e in ctx.batched_tuned() if e["key"][0] == W.DT_F64][0]
    assert t64["ms"][0] == -1 and t64["ms"][1] > 0 and t64["ms"][2] > 0
    with pytest.raises(pkg.Gpl1Error) as ei:
        run_batch(ctx, p64, W.DT_F64, r64, pkg.TILE_SMALL)
    assert ei.value.status == 7
    del ctx
