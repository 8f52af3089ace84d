"""FP64-accurate Fourier chains in FP32-pair arithmetic (llg_opts.chain_arith =
LLG_CHAIN_F32X2): the true residuals of every GMRES cycle and the step's right-hand side.

* Element-wise: the FP32-pair saddle matvec (llg_saddle_apply_f32x2) against the oracle's
  FP64 matvec on 2D and 3D grids with non-square cells, both exchange symbols, transposed
  and not.  Tolerance 2e-13 max-norm relative: inputs enter with 47 significant bits
  (2^-47 = 7e-15), each pair sum or product adds a few 2^-48 (3.6e-15) of its operands'
  magnitudes, and a value passes about 2 log2(n) butterfly levels per axis and the nodal
  terms; the FP64 chain meets 1e-15, an FP32 chain 1e-6.
* Grids with an axis outside 64..1024 have no pair chain: the entry point reports
  LLG_ERR_UNSUPPORTED_SIZE and solves fall back to FP64 chains (same results).
* Solves and steps with pair chains against the oracle at the tolerances of the FP64 path
  (solutions 1e-8, steps 1e-10), with the same GMRES iteration and restart counts as with
  FP64 chains, and tight solves (rtol 1e-12) still reaching the 1e-12 length drift.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2607_15290_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2607_15290_b300 as L  # noqa: E402

TOL_MATVEC = 2e-13


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def gpu(a, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture
def oracle_fft():
    O.set_transform(O.FFT)
    yield
    O.set_transform(O.DFT)


GRIDS = [
    ((64, 64), (1.0, 1.0)),
    ((128, 64), (1.0, 2.0)),
    ((1024, 64), (2 * np.pi, 2 * np.pi)),
    ((64, 64, 64), (1.0, 1.0, 1.0)),
    ((64, 128, 64), (1.0, 0.5, 2.0)),
]


@pytest.mark.parametrize("n,Lc", GRIDS, ids=[str(g[0]) for g in GRIDS])
@pytest.mark.parametrize("exchange", [0, 1], ids=["spectral", "fd2"])
def test_pair_matvec_vs_oracle(oracle_fft, n, Lc, exchange):
    og = O.Grid(n, Lc)
    ctx = L.Context(n, Lc)
    m = I.random_unit(n, seed=131) * 1.1
    x = I.random_saddle_vector(n, seed=132)
    for theta, transpose in ((0.5, False), (1.0, True)):
        po = O.Params(alpha=0.2, k=2e-3, theta=theta, lam=0.5, exchange=exchange)
        pl = L.Params(alpha=0.2, k=2e-3, theta=theta, lam=0.5, exchange=exchange)
        ref = O.saddle_apply(og, po, m, x, transpose=transpose)
        got = host(L.llg_saddle_apply_f32x2(ctx, pl, gpu(m), gpu(x), transpose=transpose))
        e64 = rel(host(L.llg_saddle_apply(ctx, pl, gpu(m), gpu(x), transpose=transpose)), ref)
        err = rel(got, ref)
        print(f"{n} ex={exchange} T={transpose}: pair {err:.2e}  fp64 {e64:.2e}")
        assert err <= TOL_MATVEC, (theta, transpose, err)
        # genuinely more accurate than FP32 arithmetic
        assert err <= 1e-9
    ctx.close()


def test_pair_matvec_full_size_128cube(oracle_fft):
    """The 128^3 workload's field and a random saddle vector, in the launch configuration
    the midpoint benchmark uses (autotuned shapes)."""
    n = (128, 128, 128)
    og = O.Grid(n)
    ctx = L.Context(n)
    ctx.autotune()
    m = I.smooth3d(n)
    x = I.random_saddle_vector(n, seed=133)
    alpha = 0.1
    k = 4 * 2 * alpha / ((1 + alpha ** 2) * 3 * (math.pi * 128) ** 2)
    po = O.Params(alpha=alpha, k=k, theta=0.5, lam=0.5, h=(0.0, 0.0, 0.5))
    pl = L.Params(alpha=alpha, k=k, theta=0.5, lam=0.5, h_ext=(0.0, 0.0, 0.5))
    ref = O.saddle_apply(og, po, m, x)
    err = rel(host(L.llg_saddle_apply_f32x2(ctx, pl, gpu(m), gpu(x))), ref)
    print(f"128^3 pair matvec {err:.2e}")
    assert err <= TOL_MATVEC
    ctx.close()


def test_unsupported_sizes_report_and_solves_fall_back():
    n = (32, 32)
    ctx = L.Context(n)
    pl = L.Params(alpha=0.1, k=1e-4, theta=1.0, lam=0.5, h_ext=(0.0, 0.0, 0.5))
    m = gpu(I.smooth2d(n))
    x = gpu(I.random_saddle_vector(n, seed=134))
    with pytest.raises(L.LLGError) as ei:
        L.llg_saddle_apply_f32x2(ctx, pl, m, x)
    assert "64..1024" in str(ei.value)
    outs = []
    for ch in (L.CHAIN_FP64, L.CHAIN_F32X2):
        mn, xo, info = L.llg_step_euler(ctx, pl, L.Opts(rtol=1e-10, chain_arith=ch), m)
        outs.append((host(mn), info["iters"]))
    assert outs[0][1] == outs[1][1]
    assert np.array_equal(outs[0][0], outs[1][0])
    ctx.close()


@pytest.mark.parametrize("precision", [L.PREC_FP64, L.PREC_FP32_FLEX], ids=["fp64", "fp32flex"])
def test_euler_64_pairs_vs_oracle_same_counts(precision):
    n = (64, 64)
    alpha, k = 0.1, (1 / 64) ** 2
    m0 = I.smooth2d(n)
    og = O.Grid(n)
    po = O.Params(alpha=alpha, k=k, theta=1.0, lam=0.5, h=(0.0, 0.0, 0.5))
    mo, xo, _ = O.step_euler(og, po, O.Opts(rtol=1e-13, restart=30), m0)
    ctx = L.Context(n)
    pl = L.Params(alpha=alpha, k=k, theta=1.0, lam=0.5, h_ext=(0.0, 0.0, 0.5))
    counts = []
    for ch in (L.CHAIN_FP64, L.CHAIN_F32X2):
        m, x, info = L.llg_step_euler(ctx, pl, L.Opts(restart=30, rtol=1e-10, precision=precision, chain_arith=ch),
                                      gpu(m0))
        assert rel(host(x), xo) <= 1e-8, (ch, info)
        assert float(np.abs(host(m) - mo).max()) <= 1e-10
        assert info["rel_res_true"] <= 1e-10
        counts.append((info["iters"], info["restarts"]))
    assert counts[0] == counts[1], counts
    ctx.close()


def test_stiff_restarted_solve_pairs():
    """Sec. 4.5 stiff system (the Sec. 4.3 field on (0, 2 pi)^2, 128^2, fixed k = 1e-2, seeded
    Gaussian right-hand side, GMRES(50), several restarts per solve, so many pair true
    residuals): the solution (rtol 1e-12) matches the oracle's to 1e-8, and at rtol 1e-8 the
    iteration count equals the FP64 chains' within one per restart cycle."""
    n = (128, 128)
    k = 1e-2
    m, _ = I.manufactured2d(n, 0.0, 0.2)
    b = I.gaussian_rhs(n, 20260724)
    O.set_transform(O.FFT)
    try:
        g = O.Grid(n, (2 * np.pi, 2 * np.pi))
        po = O.Params(alpha=0.2, k=k, theta=1.0, lam=0.5)
        x_ref, _ = O.gmres_solve(g, po, O.Opts(restart=50, rtol=1e-12, max_iters=20000), m, b)
    finally:
        O.set_transform(O.DFT)
    ctx = L.Context(n, (2 * np.pi, 2 * np.pi))
    pl = L.Params(alpha=0.2, k=k, theta=1.0, lam=0.5)
    gm, gb = gpu(m), gpu(b)
    for prec in (L.PREC_FP64, L.PREC_FP32_FLEX):
        x, info = L.llg_gmres_solve(ctx, pl, L.Opts(restart=50, rtol=1e-12, max_iters=20000, precision=prec,
                                                    chain_arith=L.CHAIN_F32X2), gm, gb)
        assert info["rel_res_true"] <= 1e-12, (prec, info)
        assert rel(host(x), x_ref) <= 1e-8, (prec, info)
    runs = []
    for ch in (L.CHAIN_FP64, L.CHAIN_F32X2):
        _, info = L.llg_gmres_solve(ctx, pl, L.Opts(restart=50, rtol=1e-8, max_iters=20000, chain_arith=ch), gm, gb)
        runs.append(info)
    cycles = -(-runs[0]["iters"] // 50)
    assert runs[0]["restarts"] >= 3, runs[0]
    assert abs(runs[0]["iters"] - runs[1]["iters"]) <= cycles, runs
    ctx.close()


@pytest.mark.parametrize("gs", [L.GS_FP64, L.GS_F32X2], ids=["gs_fp64", "gs_f32x2"])
def test_midpoint_64cube_pairs(gs):
    """Three midpoint steps of a 64^3 smooth field (4x the explicit limit): pair chains
    against FP64 chains (same Picard and GMRES counts, fields within 1e-11) and against the
    oracle's steps (1e-10); a tight step (rtol 1e-12) keeps the length drift within 1e-12."""
    n = (64, 64, 64)
    alpha = 0.1
    k = 4 * 2 * alpha / ((1 + alpha ** 2) * 3 * (math.pi * 64) ** 2)
    m0 = I.smooth3d(n)
    pl = L.Params(alpha=alpha, k=k, theta=0.5, lam=0.5, h_ext=(0.0, 0.0, 0.5))
    ctx = L.Context(n)
    runs = []
    for ch in (L.CHAIN_FP64, L.CHAIN_F32X2):
        o = L.Opts(restart=30, rtol=1e-10, picard_tol=1e-10, precision=L.PREC_FP32_FLEX, gs_arith=gs, chain_arith=ch)
        m, v = gpu(m0), None
        infos = []
        for _ in range(3):
            m, x, info = L.llg_step_midpoint(ctx, pl, o, m, v)
            v = x[:3].clone()
            infos.append((info["picard_iters"], info["iters"]))
        runs.append((host(m), infos))
    assert runs[0][1] == runs[1][1], (runs[0][1], runs[1][1])
    assert float(np.abs(runs[0][0] - runs[1][0]).max()) <= 1e-11
    O.set_transform(O.FFT)
    try:
        og = O.Grid(n)
        po = O.Params(alpha=alpha, k=k, theta=0.5, lam=0.5, h=(0.0, 0.0, 0.5))
        mo = O.run_midpoint(og, po, O.Opts(rtol=1e-12, picard_tol=1e-12, restart=30), m0, 3)[0][-1]
    finally:
        O.set_transform(O.DFT)
    assert float(np.abs(runs[1][0] - mo).max()) <= 1e-10
    o = L.Opts(restart=30, rtol=1e-12, picard_tol=1e-12, precision=L.PREC_FP32_FLEX, gs_arith=gs,
               chain_arith=L.CHAIN_F32X2)
    _, _, info = L.llg_step_midpoint(ctx, pl, o, gpu(m0), None)
    assert info["max_len_drift"] <= 1e-12, info
    ctx.close()
