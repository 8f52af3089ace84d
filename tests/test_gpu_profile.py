"""Live per-class timing (llg_profile_begin/end), which the bench's roofline figures use:
for a GMRES solve that ends in one cycle, the Arnoldi class reports three launches per
Arnoldi step and exactly the algorithmic bytes and flops of the steps taken (steps queued
after the cycle stopped are left out), with a positive device time.
"""
import pytest

from paper_2607_15290_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2607_15290_b300 as L  # noqa: E402


@pytest.mark.parametrize("precision", [L.PREC_FP32_FLEX, L.PREC_FP64], ids=["fp32flex", "fp64"])
def test_arnoldi_profile_counts(precision):
    n = (32, 32, 32)
    ctx = L.Context(n)
    prm = L.Params(alpha=0.1, k=2e-4, theta=0.5, lam=0.5, h_ext=(0.0, 0.0, 0.5))
    m = torch.tensor(I.smooth3d(n), device="cuda")
    b = L.llg_saddle_apply(ctx, prm, m, torch.tensor(I.random_saddle_vector(n, seed=9), device="cuda"))
    # rtol 1e-4: one cycle, also for the flexible solver (whose cycles aim at 1e-5)
    opts = L.Opts(restart=30, rtol=1e-4, precision=precision)
    ctx.profile_begin("arnoldi")
    _, info = L.llg_gmres_solve(ctx, prm, opts, m, b)
    prof = ctx.profile_end()
    assert info["restarts"] == 1, info
    jd = info["iters"]
    nu = 4 * n[0] * n[1] * n[2]
    assert prof["launches"] == 3 * jd
    assert prof["bytes"] == pytest.approx(sum(8.0 * nu * (3 * (j + 1) + 5) for j in range(jd)), rel=1e-12)
    assert prof["flops"] == pytest.approx(sum(nu * (8.0 * (j + 1) + 2.0) for j in range(jd)), rel=1e-12)
    assert prof["ms"] > 0.0
    ctx.close()
