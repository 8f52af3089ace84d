"""The cluster plan of 3D FP32 Fourier round trips (x and y transforms of each z-plane in
one thread-block cluster, three HBM passes) against the five-pass plan and the oracle.

FP32 applications are compared element by element with the oracle's FP64 application at
2e-5 (the FP32 tolerance used throughout) and with each other at 1e-6 (two FP32
evaluations of the same transforms in a different order); flexible GMRES solves with the
FP32 application and inner matvec under either plan reach the oracle's solution to 1e-8.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2607_15290_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2607_15290_b300 as L  # noqa: E402


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def apply_f32(ctx, prm, m, p, plan):
    ctx.set_pass_plan(plan)
    z = L.llg_ffthss_apply_f32(ctx, prm, torch.tensor(m, dtype=torch.float32, device="cuda"),
                               torch.tensor(p, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    return z.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n", [(128, 128, 128), (128, 128, 32), (256, 256, 16)], ids=["128cube", "128x128x32",
                                                                                       "256x256x16"])
def test_cluster_plan_apply_matches_oracle(n):
    alpha = 0.1
    k = 4 * 2 * alpha / ((1 + alpha ** 2) * 3 * (math.pi * n[0]) ** 2)
    m = I.smooth3d(n)
    p = I.random_saddle_vector(n, seed=141)
    O.set_transform(O.FFT)
    try:
        ref = O.ffthss_apply(O.Grid(n), O.Params(alpha=alpha, k=k, theta=0.5, lam=0.5), m, p)
    finally:
        O.set_transform(O.DFT)
    ctx = L.Context(n)
    prm = L.Params(alpha=alpha, k=k, theta=0.5, lam=0.5)
    zc = apply_f32(ctx, prm, m, p, L.PLAN_CLUSTER)
    zf = apply_f32(ctx, prm, m, p, L.PLAN_FIVE)
    assert rel(zc, ref) <= 2e-5 and rel(zf, ref) <= 2e-5, (rel(zc, ref), rel(zf, ref))
    assert rel(zc, zf) <= 1e-6, rel(zc, zf)
    ctx.close()


def test_cluster_plan_256cube_against_five_pass_plan():
    n = (256, 256, 256)
    ctx = L.Context(n)
    prm = L.Params(alpha=0.1, k=1e-6, theta=0.5, lam=0.5)
    m = I.smooth3d(n)
    p = I.random_saddle_vector(n, seed=142)
    zc = apply_f32(ctx, prm, m, p, L.PLAN_CLUSTER)
    zf = apply_f32(ctx, prm, m, p, L.PLAN_FIVE)
    assert np.all(np.isfinite(zc))
    assert rel(zc, zf) <= 1e-6, rel(zc, zf)
    ctx.close()


@pytest.mark.parametrize("plan", [L.PLAN_CLUSTER, L.PLAN_FIVE], ids=["cluster", "five"])
def test_flexible_solve_under_each_plan_matches_oracle(plan):
    """FP32-flexible GMRES(30) on a 128 x 128 x 32 saddle system (the FGMRES preconditioner
    reads the FP64 basis, the inner matvec writes FP64: both prologue/epilogue types of the
    cluster plan), rtol 1e-10, against the oracle's FP64 GMRES at 1e-13."""
    n = (128, 128, 32)
    alpha = 0.1
    k = 4 * 2 * alpha / ((1 + alpha ** 2) * 3 * (math.pi * 128) ** 2)
    m = I.smooth3d(n)
    b = I.random_saddle_vector(n, seed=143, zero_r=True)
    O.set_transform(O.FFT)
    try:
        x_ref, _ = O.gmres_solve(O.Grid(n), O.Params(alpha=alpha, k=k, theta=0.5, lam=0.5), O.Opts(rtol=1e-13), m, b)
    finally:
        O.set_transform(O.DFT)
    ctx = L.Context(n)
    ctx.set_pass_plan(plan)
    x, info = L.llg_gmres_solve(ctx, L.Params(alpha=alpha, k=k, theta=0.5, lam=0.5),
                                L.Opts(rtol=1e-10, precision=L.PREC_FP32_FLEX), torch.tensor(m, device="cuda"),
                                torch.tensor(b, device="cuda"))
    assert info["rel_res_true"] <= 1e-10
    assert rel(x.cpu().numpy(), x_ref) <= 1e-8, rel(x.cpu().numpy(), x_ref)
    ctx.close()
