"""The degenerate-node check (a node with |m_i| = 0 makes the saddle matrix singular, Sec.
2.4): a solve on such a field fails with LLG_ERR_DEGENERATE_NODE before any Krylov cycle, in
FP64 and FP32-flexible precision (the latter checks in the pass that makes the FP32 copy of
m, read with the solve's first scalars), and the context stays usable."""
import numpy as np
import pytest

from paper_2607_15290_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2607_15290_b300 as L  # noqa: E402


@pytest.mark.parametrize("precision", [L.PREC_FP64, L.PREC_FP32_FLEX], ids=["fp64", "fp32flex"])
@pytest.mark.parametrize("bad", ["zero", "nan"])
def test_degenerate_node_rejected_then_solve(precision, bad):
    n = (64, 64)
    ctx = L.Context(n)
    pl = L.Params(alpha=0.1, k=1e-4, theta=1.0, lam=0.5)
    m = I.smooth2d(n)
    b = I.random_saddle_vector(n, seed=151)
    mb = m.copy()
    mb[:, 17, 9] = 0.0 if bad == "zero" else np.nan
    opts = L.Opts(restart=30, rtol=1e-10, precision=precision, gs_arith=L.GS_F32X2, chain_arith=L.CHAIN_F32X2)
    with pytest.raises(L.LLGError) as ei:
        L.llg_gmres_solve(ctx, pl, opts, torch.tensor(mb, device="cuda"), torch.tensor(b, device="cuda"))
    assert ei.value.status == 5 and "|m_i| = 0" in str(ei.value)
    x, info = L.llg_gmres_solve(ctx, pl, opts, torch.tensor(m, device="cuda"), torch.tensor(b, device="cuda"))
    torch.cuda.synchronize()
    assert info["rel_res_true"] <= 1e-10 and np.isfinite(x.cpu().numpy()).all()
    ctx.close()
