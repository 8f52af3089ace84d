"""Random right-hand-side mesh study of Sec. 4.5 on the GPU against the oracle.

The velocity right-hand side is a seeded normalised Gaussian vector (seed 20260724, the
first of the paper's seeds; not the paper's NumPy vector), the multiplier part zero, on the
Sec. 4.3 field (manufactured solution at t = 0 on (0, 2 pi)^2, alpha = 0.2, lambda = 0.5),
FFT--HSS GMRES(50).  Two regimes: bounded stiffness k N^2 = 10.24 (13.31x the explicit limit)
and fixed k = 1e-2, where the count grows with N and GMRES(50) restarts several times per
solve.  The solution (FP64 and FP32-flexible, rtol 1e-12) matches the oracle's to 1e-8
relative; at the paper's rtol 1e-8 the FP64 iteration count equals the oracle's within the
spread that classical vs modified Gram--Schmidt leaves in a restarted run (+-1 per restart
cycle, at least +-1).
"""
import numpy as np
import pytest

import oracle as O
from paper_2607_15290_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2607_15290_b300 as L  # noqa: E402

CASES = [(64, 10.24 / 64 ** 2), (128, 10.24 / 128 ** 2), (64, 1e-2), (128, 1e-2)]


@pytest.mark.parametrize("N,k", CASES, ids=["64-bounded", "128-bounded", "64-fixed", "128-fixed"])
def test_random_rhs_solve_matches_oracle(N, k):
    n = (N, N)
    m, _ = I.manufactured2d(n, 0.0, 0.2)
    b = I.gaussian_rhs(n, 20260724)
    O.set_transform(O.FFT)
    try:
        g = O.Grid(n, (2 * np.pi, 2 * np.pi))
        po = O.Params(alpha=0.2, k=k, theta=1.0, lam=0.5)
        x_ref, info_t = O.gmres_solve(g, po, O.Opts(restart=50, rtol=1e-12, max_iters=20000), m, b)
        _, info_o = O.gmres_solve(g, po, O.Opts(restart=50, rtol=1e-8, max_iters=20000), m, b)
    finally:
        O.set_transform(O.DFT)
    assert info_t.converged and info_o.converged
    ctx = L.Context(n, (2 * np.pi, 2 * np.pi))
    pl = L.Params(alpha=0.2, k=k, theta=1.0, lam=0.5)
    gm, gb = torch.tensor(m, device="cuda"), torch.tensor(b, device="cuda")
    for prec in (L.PREC_FP64, L.PREC_FP32_FLEX):
        x, info = L.llg_gmres_solve(ctx, pl, L.Opts(restart=50, rtol=1e-12, max_iters=20000, precision=prec), gm, gb)
        assert info["rel_res_true"] <= 1e-12, (prec, info)
        got = x.cpu().numpy()
        assert float(np.abs(got - x_ref).max() / np.abs(x_ref).max()) <= 1e-8, (prec, info)
    _, info = L.llg_gmres_solve(ctx, pl, L.Opts(restart=50, rtol=1e-8, max_iters=20000), gm, gb)
    cycles = -(-info_o.iters // 50)
    assert abs(info["iters"] - info_o.iters) <= max(1, cycles), (info["iters"], info_o.iters)
    if N == 128 and k == 1e-2:
        assert info["restarts"] >= 3, info          # the heavily restarted regime
    ctx.close()
