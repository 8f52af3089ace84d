"""Parity at the workloads' full sizes, in the launch configuration bench.py times
(autotuned axis-pass shapes).

* Element-wise: FFT--HSS applies (FP64 and FP32) and saddle matvecs at 1024^2, 128^3 and
  256^3 against the oracle, which runs its radix-2 FFT mode there (pinned against the
  naive DFT on small grids); tolerances as in test_gpu_parity (1e-12 FP64, 2e-5 FP32).
* Properties that hold at any size: for the 128^3 midpoint workload and the 1024^2
  midpoint workload (smooth and broadband fields) solved tightly, nodal length drift
  <= 1e-12, the exact discrete dissipation identity, the energy against the oracle's.
* Element-wise at the 128^3 workload: its first Picard system solved on the GPU (FP32-flexible
  and FP64, rtol 1e-10) against the oracle's FP64 GMRES solution (rtol 1e-12) to 1e-8.
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
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def gpu(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture
def oracle_fft():
    O.set_transform(O.FFT)
    yield
    O.set_transform(O.DFT)


def k_explicit(alpha, n, dim):
    """explicit exchange limit 2 alpha / (Chat max|xi|^2) on the unit cell, spectral symbol"""
    return 2 * alpha / ((1 + alpha ** 2) * dim * (math.pi * n) ** 2)


def workload(n):
    """(alpha, k) of the 1024^2 midpoint workload (13.3x the limit) and of the 128^3 / 256^3
    one (4x)"""
    if len(n) == 2:
        return 0.02, 13.3 * k_explicit(0.02, n[0], 2)
    return 0.1, 4 * k_explicit(0.1, n[0], 3)


@pytest.mark.parametrize("n", [(1024, 1024), (128, 128, 128)], ids=["1024sq", "128cube"])
def test_full_size_apply_and_matvec(oracle_fft, n):
    og = O.Grid(n)
    ctx = L.Context(n)
    ctx.autotune()
    m = I.smooth2d(n) if len(n) == 2 else I.smooth3d(n)
    p = I.random_saddle_vector(n, seed=121)
    alpha, k = workload(n)
    po = O.Params(alpha=alpha, k=k, theta=0.5, lam=0.5, h=(0.0, 0.0, 0.5))
    pl = L.Params(alpha=alpha, k=k, theta=0.5, lam=0.5, h_ext=(0.0, 0.0, 0.5))
    gm, gp = gpu(m), gpu(p)
    ref = O.ffthss_apply(og, po, m, p)
    assert rel(host(L.llg_ffthss_apply(ctx, pl, gm, gp)), ref) <= 1e-12
    got32 = host(L.llg_ffthss_apply_f32(ctx, pl, gpu(m, torch.float32), gpu(p, torch.float32)))
    assert rel(got32, ref) <= 2e-5
    ref_s = O.saddle_apply(og, po, m, p)
    assert rel(host(L.llg_saddle_apply(ctx, pl, gm, gp)), ref_s) <= 1e-12
    ctx.close()


def test_full_size_256cube_apply(oracle_fft):
    n = (256, 256, 256)
    og = O.Grid(n)
    ctx = L.Context(n)
    ctx.autotune(fp64=False, fp32=True)
    m = I.smooth3d(n)
    p = I.random_saddle_vector(n, seed=122)
    alpha, k = workload(n)
    po = O.Params(alpha=alpha, k=k, theta=0.5, lam=0.5)
    pl = L.Params(alpha=alpha, k=k, theta=0.5, lam=0.5)
    ref = O.ffthss_apply(og, po, m, p)
    got = host(L.llg_ffthss_apply_f32(ctx, pl, gpu(m, torch.float32), gpu(p, torch.float32)))
    assert rel(got, ref) <= 2e-5
    # FP64 apply and saddle matvec at the full 256^3 size as well
    gm, gp = gpu(m), gpu(p)
    assert rel(host(L.llg_ffthss_apply(ctx, pl, gm, gp)), ref) <= 1e-12
    assert rel(host(L.llg_saddle_apply(ctx, pl, gm, gp)), O.saddle_apply(og, po, m, p)) <= 1e-12
    ctx.close()


def midpoint_checks(ctx, og, po, pl, m0, steps, opts):
    mg, vg = gpu(m0), None
    for _ in range(steps):
        e_prev = O.energy(og, po, host(mg))
        mg, xg, info = L.llg_step_midpoint(ctx, pl, opts, mg, vg)
        vg = xg[:3].contiguous()
        assert info["rel_res_true"] <= opts.rtol, info
        assert info["max_len_drift"] <= 1e-12, info
        assert abs(info["energy_before"] - e_prev) <= 1e-11 * abs(e_prev)
        assert abs(info["energy_after"] - O.energy(og, po, host(mg))) <= 1e-11 * abs(e_prev)
        assert abs(info["dissipation_residual"]) <= 1e-9 * abs(e_prev)
    return mg


def picard_system(og, po, m):
    """The first Picard system of a midpoint step from rest (v^{n-1/2} = 0, so mhat^0 = m^n):
    theta = 1/2, blocks from m^n, b = (Chat Lap_N m^n + (1 + alpha^2) h, 0) (Sec. 3.3 eqs.
    (C-N), (hatm)); the right-hand side is the oracle's."""
    s = 1 + po.alpha ** 2
    b = np.zeros((4,) + og.shape)
    lap = np.stack([-O.neg_laplacian(og, m[c]) for c in range(3)])
    b[:3] = s * lap + s * O.h_low(og, po, m)
    return b


def test_full_size_midpoint_128cube(oracle_fft):
    """The bench workload (FP32-flexible FGMRES(30)) at full size.  Solved tightly, the
    invariants hold; and the first Picard system of its first step, solved on the GPU in
    FP32-flexible and in FP64 GMRES(30) at the workload's rtol 1e-10 (Gram--Schmidt passes in
    FP64 and in FP32-pair arithmetic), matches the oracle's FP64 GMRES solution at rtol 1e-12
    element by element to 1e-8."""
    n = (128, 128, 128)
    og = O.Grid(n)
    ctx = L.Context(n)
    ctx.autotune()
    alpha, k = workload(n)
    po = O.Params(alpha=alpha, k=k, theta=0.5, lam=0.5, h=(0.0, 0.0, 0.5))
    pl = L.Params(alpha=alpha, k=k, theta=0.5, lam=0.5, h_ext=(0.0, 0.0, 0.5))
    m0 = I.smooth3d(n)
    tight = L.Opts(restart=30, rtol=1e-12, picard_tol=1e-12, picard_max=50, precision=L.PREC_FP32_FLEX,
                   diagnostics=1)
    midpoint_checks(ctx, og, po, pl, m0, 2, tight)
    b = picard_system(og, po, m0)
    x_ref, info_o = O.gmres_solve(og, po, O.Opts(restart=30, rtol=1e-12, max_iters=600), m0, b)
    assert info_o.converged
    gm, gb = gpu(m0), gpu(b)
    for prec in (L.PREC_FP32_FLEX, L.PREC_FP64):
        for gs in (L.GS_FP64, L.GS_F32X2):
            x, info = L.llg_gmres_solve(ctx, pl, L.Opts(restart=30, rtol=1e-10, max_iters=600, precision=prec,
                                                        gs_arith=gs), gm, gb)
            assert info["rel_res_true"] <= 1e-10, (prec, gs, info)
            assert rel(host(x), x_ref) <= 1e-8, (prec, gs, rel(host(x), x_ref))
    ctx.close()


@pytest.mark.parametrize("field", ["smooth", "broadband"])
def test_full_size_midpoint_1024sq(oracle_fft, field):
    """The 1024^2 FP64 midpoint workload (alpha 0.02, 13.3x the explicit limit), both fields."""
    n = (1024, 1024)
    og = O.Grid(n)
    ctx = L.Context(n)
    ctx.autotune(fp64=True, fp32=False)
    alpha, k = workload(n)
    po = O.Params(alpha=alpha, k=k, theta=0.5, lam=0.5)
    pl = L.Params(alpha=alpha, k=k, theta=0.5, lam=0.5)
    m0 = I.smooth2d(n) if field == "smooth" else I.broadband(n, seed=20260725)
    opts = L.Opts(restart=30, rtol=1e-12, picard_tol=1e-12, picard_max=60, diagnostics=1)
    midpoint_checks(ctx, og, po, pl, m0, 2, opts)
    ctx.close()
