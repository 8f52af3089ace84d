"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Tolerances (from the arithmetic and the stated targets):
  * FP64 preconditioner / matvec / fused operator: max-norm relative error 1e-12
    (FFT rounding grows like eps * log2(N_g); 1e-12 leaves a ~50x margin);
  * FP32 preconditioner: 2e-5 (FP32 eps 6e-8 times the transform depth and the
    conditioning of the shifted symbol);
  * solutions at GMRES rtol 1e-10: relative error 1e-8 against the oracle's
    dense-LU or tight GMRES solution; time steps the same; midpoint nodal length
    drift 1e-12.
Grid sizes span several column tiles, row-pair groups with a ragged last block,
non-square cells and the 1024-point line length (the largest supported).
"""
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


def gpu(a, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def prm_pair(alpha=0.2, k=1e-2, theta=1.0, lam=0.5, h=(0.0, 0.0, 0.0), exchange=0):
    return (O.Params(alpha=alpha, k=k, theta=theta, lam=lam, h=h, exchange=exchange),
            L.Params(alpha=alpha, k=k, theta=theta, lam=lam, h_ext=h, exchange=exchange))


GRIDS = [
    ((16, 8), (1.0, 2.0)),
    ((64, 32), (1.0, 1.0)),
    ((1024, 8), (1.0, 1.0)),
    ((8, 1024), (2 * np.pi, 2 * np.pi)),
    ((2, 4), (1.0, 1.0)),
    ((8, 4, 16), (1.0, 1.0, 1.0)),
    ((8, 64, 32), (1.0, 0.5, 2.0)),      # 1024 row pairs: ragged last row-pair block
    ((16, 16, 16), (2 * np.pi,) * 3),
]


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.device("cuda")


@pytest.mark.parametrize("n,Lc", GRIDS, ids=[str(g[0]) for g in GRIDS])
@pytest.mark.parametrize("exchange", [0, 1], ids=["spectral", "fd2"])
def test_apply_fp64(dev, n, Lc, exchange):
    og = O.Grid(n, Lc)
    ctx = L.Context(n, Lc)
    m = I.random_unit(n, seed=101)
    p = I.random_saddle_vector(n, seed=102)
    for theta, transpose in ((1.0, False), (0.5, True)):
        po, pl = prm_pair(alpha=0.1, k=3e-3, theta=theta, exchange=exchange)
        ref = O.ffthss_apply(og, po, m, p, transpose=transpose)
        got = host(L.llg_ffthss_apply(ctx, pl, gpu(m), gpu(p), transpose=transpose))
        assert rel(got, ref) <= 1e-12, (theta, transpose)


@pytest.mark.parametrize("n,Lc", GRIDS[:6], ids=[str(g[0]) for g in GRIDS[:6]])
def test_apply_fp32(dev, n, Lc):
    og = O.Grid(n, Lc)
    ctx = L.Context(n, Lc)
    m = I.random_unit(n, seed=103)
    p = I.random_saddle_vector(n, seed=104)
    po, pl = prm_pair(alpha=0.1, k=3e-3)
    for transpose in (False, True):
        ref = O.ffthss_apply(og, po, m, p, transpose=transpose)
        got = host(L.llg_ffthss_apply_f32(ctx, pl, gpu(m, torch.float32), gpu(p, torch.float32), transpose=transpose))
        assert rel(got, ref) <= 2e-5


@pytest.mark.parametrize("n,Lc", GRIDS, ids=[str(g[0]) for g in GRIDS])
def test_saddle_and_fused_operator(dev, n, Lc):
    og = O.Grid(n, Lc)
    ctx = L.Context(n, Lc)
    m = I.random_unit(n, seed=105) * 1.1
    x = I.random_saddle_vector(n, seed=106)
    po, pl = prm_pair(alpha=0.2, k=2e-3, theta=0.5)
    for transpose in (False, True):
        ref = O.saddle_apply(og, po, m, x, transpose=transpose)
        got = host(L.llg_saddle_apply(ctx, pl, gpu(m), gpu(x), transpose=transpose))
        assert rel(got, ref) <= 1e-12
    ref = O.ffthss_apply(og, po, m, O.saddle_apply(og, po, m, x))
    got = host(L.llg_precond_saddle_apply(ctx, pl, gpu(m), gpu(x)))
    assert rel(got, ref) <= 1e-12


@pytest.mark.parametrize("n", [(8, 8), (4, 4, 4), (32, 16)])
@pytest.mark.parametrize("precision", [L.PREC_FP64, L.PREC_FP32_FLEX], ids=["fp64", "fp32flex"])
def test_gmres_vs_dense_lu(dev, n, precision):
    og = O.Grid(n)
    ctx = L.Context(n)
    m = I.random_unit(n, seed=107)
    b = I.random_saddle_vector(n, seed=108, zero_r=True)
    po, pl = prm_pair(alpha=0.1, k=5e-3, theta=1.0, h=(0, 0, 0.5))
    if og.nodes <= 256:
        A = O.saddle_dense(og, po, m)
        ref = np.linalg.solve(A, b.ravel()).reshape(b.shape)
    else:
        ref, info = O.gmres_solve(og, po, O.Opts(rtol=1e-13), m, b)
        assert info.converged
    x, info = L.llg_gmres_solve(ctx, pl, L.Opts(rtol=1e-10, precision=precision), gpu(m), gpu(b))
    assert info["rel_res_true"] <= 1e-10
    assert rel(host(x), ref) <= 1e-8


def test_gmres_config0_euler_system(dev):
    """One projected-Euler saddle solve of the 64x64 smooth workload (alpha 0.1, h = (0,0,0.5),
    dt = h^2), FP64 and FP32-flexible, against the oracle's tight GMRES solution."""
    n = (64, 64)
    og = O.Grid(n)
    ctx = L.Context(n)
    m = I.smooth2d(n)
    k = (1.0 / 64) ** 2
    po, pl = prm_pair(alpha=0.1, k=k, theta=1.0, h=(0.0, 0.0, 0.5))
    chat = 1.01
    f = np.concatenate([-chat * np.stack([O.neg_laplacian(og, m[c]) for c in range(3)])
                        + 1.01 * np.array([0, 0, 0.5]).reshape(3, 1, 1), np.zeros((1,) + og.shape)])
    ref, oi = O.gmres_solve(og, po, O.Opts(rtol=1e-13, restart=30), m, f)
    assert oi.converged
    for prec in (L.PREC_FP64, L.PREC_FP32_FLEX):
        x, info = L.llg_gmres_solve(ctx, pl, L.Opts(rtol=1e-10, precision=prec), gpu(m), gpu(f))
        assert rel(host(x), ref) <= 1e-8, prec


def test_euler_step(dev):
    n = (64, 64)
    og = O.Grid(n)
    ctx = L.Context(n)
    m = I.smooth2d(n)
    po, pl = prm_pair(alpha=0.1, k=(1.0 / 64) ** 2, h=(0.0, 0.0, 0.5))
    mo, xo, _ = O.step_euler(og, po, O.Opts(rtol=1e-13), m)
    mg, xg, info = L.llg_step_euler(ctx, pl, L.Opts(rtol=1e-10), gpu(m))
    assert rel(host(xg), xo) <= 1e-8
    assert rel(host(mg), mo) <= 1e-12
    assert np.abs(np.sqrt((host(mg) ** 2).sum(0)) - 1).max() <= 1e-14


@pytest.mark.parametrize("n", [(32, 16), (8, 8, 8)])
def test_midpoint_steps(dev, n):
    og = O.Grid(n)
    ctx = L.Context(n)
    m = I.smooth2d(n) if len(n) == 2 else I.smooth3d(n)
    po, pl = prm_pair(alpha=0.1, k=4e-3 if len(n) == 2 else 2e-3, theta=0.5, h=(0.0, 0.0, 0.5))
    oo = O.Opts(rtol=1e-13, picard_tol=1e-13)
    # a 1e-12 nodal-length drift needs solves at 1e-12: drift = k^2 (v^p - v^{p-1}).v^p + 2 k chi
    lo = L.Opts(rtol=1e-12, picard_tol=1e-12, diagnostics=1)
    mo, vo = m, None
    mg, vg = gpu(m), None
    for step in range(3):
        e_prev = O.energy(og, po, mo)
        mo, xo, _ = O.step_midpoint(og, po, oo, mo, vo)
        vo = xo[:3]
        mg, xg, info = L.llg_step_midpoint(ctx, pl, lo, mg, vg)
        vg = xg[:3].contiguous()
        assert rel(host(xg)[:3], xo[:3]) <= 1e-8
        assert rel(host(mg), mo) <= 1e-10
        assert info["max_len_drift"] <= 1e-12
        assert abs(info["energy_before"] - e_prev) <= 1e-11 * abs(e_prev)
        assert abs(info["energy_after"] - O.energy(og, po, mo)) <= 1e-11 * abs(e_prev)
        # exact discrete dissipation identity up to the solver tolerance (Prop. energy law)
        assert abs(info["dissipation_residual"]) <= 1e-9 * abs(e_prev)


def test_energy(dev):
    n = (32, 16)
    og = O.Grid(n, (1.0, 0.5))
    ctx = L.Context(n, (1.0, 0.5))
    m = I.smooth2d(n)
    po, pl = prm_pair(h=(0.1, 0.0, 0.5))
    assert abs(L.llg_energy(ctx, pl, gpu(m)) - O.energy(og, po, m)) <= 1e-12 * abs(O.energy(og, po, m))


def test_adjoint_step(dev):
    n = (16, 16)
    og = O.Grid(n)
    ctx = L.Context(n)
    m = I.smooth2d(n, noise=0.05)
    mbar = I.random_saddle_vector(n, seed=109)[:3]
    po, pl = prm_pair(alpha=0.1, k=2e-3, theta=0.5, h=(0.1, -0.2, 0.5))
    oo = O.Opts(rtol=1e-13, picard_tol=1e-14, picard_max=100)
    _, xo, _ = O.step_midpoint(og, po, oo, m)
    mb_o, da_o, dh_o, _ = O.adjoint_midpoint(og, po, oo, m, xo, mbar)
    mb_g, da_g, dh_g, info = L.llg_adjoint_step(ctx, pl, L.Opts(rtol=1e-12), gpu(m), gpu(xo), gpu(mbar))
    assert rel(host(mb_g), mb_o) <= 1e-8
    assert abs(da_g - da_o) <= 1e-8 * abs(da_o)
    assert np.abs(np.array(dh_g) - dh_o).max() <= 1e-8 * np.abs(dh_o).max()


def test_error_statuses(dev):
    n = (16, 16)
    ctx = L.Context(n)
    m = I.random_unit(n, seed=110)
    b = I.random_saddle_vector(n, seed=111, zero_r=True)
    _, pl = prm_pair()
    m0 = m.copy()
    m0[:, 3, 5] = 0.0
    with pytest.raises(L.LLGError) as e:
        L.llg_gmres_solve(ctx, pl, L.Opts(), gpu(m0), gpu(b))
    assert e.value.status == 5
    x, info = L.llg_gmres_solve(ctx, pl, L.Opts(max_iters=1, rtol=1e-12), gpu(m), gpu(b), raise_on_error=False)
    assert info["status"] == 3 and info["iters"] == 1
    bad = b.copy()
    bad[0, 0, 0] = np.nan
    x, info = L.llg_gmres_solve(ctx, pl, L.Opts(), gpu(m), gpu(bad), raise_on_error=False)
    assert info["status"] == 4
    # the context stays usable after errors
    x, info = L.llg_gmres_solve(ctx, pl, L.Opts(), gpu(m), gpu(b))
    assert info["status"] == 0


@pytest.mark.parametrize("n", [(64, 32, 64), (256, 16), (16, 128, 128)])
def test_autotuned_shapes_keep_parity(dev, n):
    """After llg_autotune picks launch shapes (staged or register axis passes), FP64 and FP32
    applies still match the oracle at the usual tolerances."""
    og = O.Grid(n)
    ctx = L.Context(n)
    report = ctx.autotune()
    assert "->" in report
    m = I.random_unit(n, seed=112)
    p = I.random_saddle_vector(n, seed=113)
    po, pl = prm_pair(alpha=0.1, k=1e-4, theta=0.5)
    ref = O.ffthss_apply(og, po, m, p)
    got = host(L.llg_ffthss_apply(ctx, pl, gpu(m), gpu(p)))
    assert rel(got, ref) <= 1e-12
    got32 = host(L.llg_ffthss_apply_f32(ctx, pl, gpu(m, torch.float32), gpu(p, torch.float32)))
    assert rel(got32, ref) <= 2e-5
    ref_t = O.saddle_apply(og, po, m, p, transpose=True)
    assert rel(host(L.llg_saddle_apply(ctx, pl, gpu(m), gpu(p), transpose=True)), ref_t) <= 1e-12


# Grids whose axes cover every line length with a compile-time plan (64..1024) in each
# role: x rows (nodal prologue/epilogue), y columns and z columns (forward, multiplier,
# inverse), in FP64 and FP32, before and after the autotuner picks staged shapes.
CT_GRIDS = [(128, 512, 16), (16, 8, 512), (8, 16, 1024), (256, 8, 256), (512, 256), (1024, 64), (64, 128)]


@pytest.fixture
def oracle_fft():
    O.set_transform(O.FFT)   # the textbook radix-2 FFT, pinned against the naive DFT
    yield
    O.set_transform(O.DFT)


@pytest.mark.parametrize("n", CT_GRIDS, ids=[str(g) for g in CT_GRIDS])
def test_compiled_lengths_parity(dev, oracle_fft, n):
    og = O.Grid(n)
    ctx = L.Context(n)
    m = I.random_unit(n, seed=114) * 1.05
    p = I.random_saddle_vector(n, seed=115)
    po, pl = prm_pair(alpha=0.1, k=2e-4, theta=0.5)
    gm, gp, gm32, gp32 = gpu(m), gpu(p), gpu(m, torch.float32), gpu(p, torch.float32)
    for tuned in (False, True):
        if tuned:
            assert "->" in ctx.autotune()
        for transpose in (False, True):
            ref = O.ffthss_apply(og, po, m, p, transpose=transpose)
            assert rel(host(L.llg_ffthss_apply(ctx, pl, gm, gp, transpose=transpose)), ref) <= 1e-12, (tuned, transpose)
            got32 = host(L.llg_ffthss_apply_f32(ctx, pl, gm32, gp32, transpose=transpose))
            assert rel(got32, ref) <= 2e-5, (tuned, transpose)
            ref_s = O.saddle_apply(og, po, m, p, transpose=transpose)
            assert rel(host(L.llg_saddle_apply(ctx, pl, gm, gp, transpose=transpose)), ref_s) <= 1e-12, (tuned, transpose)
        ref_f = O.ffthss_apply(og, po, m, O.saddle_apply(og, po, m, p))
        assert rel(host(L.llg_precond_saddle_apply(ctx, pl, gm, gp)), ref_f) <= 1e-12, tuned
