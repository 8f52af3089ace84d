"""Gram--Schmidt passes of flexible solves in FP32-pair arithmetic (llg_opts.gs_arith =
LLG_GS_F32X2: basis vectors after the first stored as planar FP32 pairs, about 47 significant
bits, error-free FP32 products and two-sums) against the FP64 multiply-add passes and the
oracle.  Required: the same solutions as the oracle at the stated tolerances, the same GMRES
iteration counts as the FP64 passes on the 64^2 Euler system and on the Sec. 4.3 comparison
systems, and an orthogonality max |I - V^T V| of one 30-step flexible cycle at 128^3 within
1e-12 (reported beside the FP64 passes' figure).  FP64-precision solves ignore the setting.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2607_15290_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2607_15290_b300 as L  # noqa: E402

ARITH = [L.GS_FP64, L.GS_F32X2]


def euler_system_64():
    """The 64^2 single Euler step of the smooth-field workload (alpha 0.1, h = (0,0,0.5),
    dt = h^2, GMRES(30), rtol 1e-10)."""
    n = (64, 64)
    return n, 0.1, (1 / 64) ** 2, I.smooth2d(n)


@pytest.mark.parametrize("precision", [L.PREC_FP64, L.PREC_FP32_FLEX], ids=["fp64", "fp32flex"])
def test_euler_64_same_counts_and_oracle_solution(precision):
    n, alpha, k, m0 = euler_system_64()
    og = O.Grid(n)
    po = O.Params(alpha=alpha, k=k, theta=1.0, lam=0.5, h=(0.0, 0.0, 0.5))
    mo, xo, _ = O.step_euler(og, po, O.Opts(rtol=1e-13, restart=30), m0)
    ctx = L.Context(n)
    pl = L.Params(alpha=alpha, k=k, theta=1.0, lam=0.5, h_ext=(0.0, 0.0, 0.5))
    counts = []
    for gs in ARITH:
        m, x, info = L.llg_step_euler(ctx, pl, L.Opts(restart=30, rtol=1e-10, precision=precision, gs_arith=gs),
                                      torch.tensor(m0, device="cuda"))
        torch.cuda.synchronize()
        xh = x.cpu().numpy()
        assert float(np.abs(xh - xo).max() / np.abs(xo).max()) <= 1e-8, (gs, info)
        assert float(np.abs(m.cpu().numpy() - mo).max()) <= 1e-10
        counts.append((info["iters"], info["restarts"]))
    assert counts[0] == counts[1], counts
    ctx.close()


@pytest.mark.parametrize("N", [64, 256])
def test_comparison_systems_same_counts(N):
    """Sec. 4.3 one-step Euler system (manufactured solution, alpha 0.2, k 1e-2, GMRES(50),
    FFT--HSS): at rtol 1e-8 both arithmetics take the printed 11 iterations, and at rtol
    1e-12 both reach the oracle's solution to 1e-8."""
    n = (N, N)
    alpha, k = 0.2, 1e-2
    g = O.Grid(n, (2 * np.pi, 2 * np.pi))
    m, _ = I.manufactured2d(n, 0.0, alpha)
    _, f = I.manufactured2d(n, k, alpha)
    po = O.Params(alpha=alpha, k=k, theta=1.0, lam=0.5, h_field=f)
    lap = np.stack([-O.neg_laplacian(g, m[c]) for c in range(3)])
    b = np.zeros((4,) + g.shape)
    b[:3] = (1 + alpha ** 2) * lap + (1 + alpha ** 2) * O.h_low(g, po, m)
    O.set_transform(O.FFT)
    try:
        x_ref, _ = O.gmres_solve(g, po, O.Opts(restart=50, rtol=1e-12, max_iters=4000), m, b)
    finally:
        O.set_transform(O.DFT)
    ctx = L.Context(n, (2 * np.pi, 2 * np.pi))
    pl = L.Params(alpha=alpha, k=k, theta=1.0, lam=0.5)
    gm, gb = torch.tensor(m, device="cuda"), torch.tensor(b, device="cuda")
    # restart 30 (the pair passes cover up to 32 basis vectors); 11 iterations need no restart
    counts = []
    for gs in ARITH:
        for prec in (L.PREC_FP64, L.PREC_FP32_FLEX):
            x, info = L.llg_gmres_solve(ctx, pl, L.Opts(restart=30, rtol=1e-12, precision=prec, gs_arith=gs), gm, gb)
            err = float(np.abs(x.cpu().numpy() - x_ref).max() / np.abs(x_ref).max())
            assert err <= 1e-8, (gs, prec, err, info)
        _, info = L.llg_gmres_solve(ctx, pl, L.Opts(restart=30, rtol=1e-8, gs_arith=gs), gm, gb)
        assert info["iters"] == 11, (gs, info)
        _, info = L.llg_gmres_solve(ctx, pl, L.Opts(restart=30, rtol=1e-8, gs_arith=gs, precision=L.PREC_FP32_FLEX),
                                    gm, gb)
        counts.append((info["iters"], info["restarts"]))
    assert counts[0] == counts[1], counts
    ctx.close()


def test_orthogonality_of_a_30_step_cycle_128cube():
    """One 30-step flexible cycle on the 128^3 saddle operator without preconditioner at 400x
    the explicit step limit (stiff enough that the cycle does not reach its 1e-5 reduction
    target within 30 steps), a random right-hand side, max_iters 30: the stored basis stays
    orthonormal to 1e-12 in FP32-pair arithmetic; both figures are printed.  (The first vector
    holds the final residual after the solve, so the 30 vectors after it are compared.)"""
    n = (128, 128, 128)
    alpha = 0.1
    k = 400 * 2 * alpha / ((1 + alpha ** 2) * 3 * (math.pi * 128) ** 2)
    ctx = L.Context(n)
    pl = L.Params(alpha=alpha, k=k, theta=0.5, lam=0.5, h_ext=(0.0, 0.0, 0.5))
    m0 = torch.tensor(I.smooth3d(n), device="cuda")
    b = torch.tensor(I.random_saddle_vector(n, seed=131), device="cuda")
    res = {}
    for gs in ARITH:
        _, info = L.llg_gmres_solve(ctx, pl, L.Opts(restart=30, rtol=1e-30, max_iters=30, gs_arith=gs,
                                                    precision=L.PREC_FP32_FLEX, preconditioner=L.PC_NONE),
                                    m0, b, raise_on_error=False)
        assert info["iters"] == 30 and info["status"] == 3, info   # NOT_CONVERGED after the one cycle
        res[gs] = ctx.krylov_orthogonality()
    print("max |I - V^T V| over a 30-step flexible cycle at 128^3: FP64 %.3e (%d vectors), FP32 pairs %.3e (%d vectors)"
          % (res[L.GS_FP64][0], res[L.GS_FP64][1], res[L.GS_F32X2][0], res[L.GS_F32X2][1]))
    assert res[L.GS_FP64][1] == 30 and res[L.GS_F32X2][1] == 30
    assert res[L.GS_FP64][0] <= 1e-12 and res[L.GS_F32X2][0] <= 1e-12
    ctx.close()
