"""Gradients of L = 1/2 sum_i |m_i(T) - m_target,i|^2 through midpoint trajectories on the GPU
(adjoint of the converged midpoint map, transposed FFT--HSS preconditioner, uniform
checkpointing) against the CPU oracle's adjoint and against central finite differences.

Tolerances: against the oracle 1e-8 relative (both sides solve to ~1e-13); against central
differences with step 1e-6 the target is 1e-6 relative (the FD truncation error is O(eps^2);
the finite-difference forwards use fixed iteration counts, see FD_OPTS).
"""
import numpy as np
import pytest

import oracle as O
from paper_2607_15290_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2607_15290_b300 as L  # noqa: E402
from paper_2607_15290_b300.autograd import midpoint_trajectory  # noqa: E402


def loss_and_grads(ctx, m0, tgt, alpha, h, k, nsteps, opts, checkpoint):
    a = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    hh = torch.tensor(h, dtype=torch.float64, requires_grad=True)
    m = m0.clone().requires_grad_(True)
    mT = midpoint_trajectory(ctx, m, a, hh, k, nsteps, opts=opts, checkpoint=checkpoint)
    loss = 0.5 * ((mT - tgt) ** 2).sum()
    loss.backward()
    return float(loss.detach()), float(a.grad), hh.grad.numpy().copy(), m.grad.detach()


# Finite-difference forwards run a FIXED number of GMRES and Picard iterations (tolerances
# below reach), so the discrete forward map is a smooth function of the inputs: with
# tolerance-based stopping the +eps and -eps runs stop at different iterates and their
# ~1e-13 solver errors, divided by 2 eps, swamp a 1e-6 comparison.  The fixed counts
# converge to rounding level for these steps.
FD_OPTS = L.Opts(rtol=1e-16, max_iters=40, restart=40, picard_tol=1e-300, picard_max=6)


def forward_mT(ctx, m0, alpha, h, k, nsteps, opts=FD_OPTS):
    prm = L.Params(alpha=alpha, k=k, theta=0.5, lam=0.5, h_ext=tuple(h))
    m, vprev = m0, None
    for _ in range(nsteps):
        m, x, info = L.llg_step_midpoint(ctx, prm, opts, m, vprev, raise_on_error=False)
        assert info["status"] in (0, 3), info            # 3: the fixed iteration counts ran out
        assert info["rel_res_true"] <= 1e-13, info
        vprev = x[:3].contiguous()
    return m


def central_difference(mp, mm, tgt, eps):
    """(L(m+) - L(m-)) / (2 eps) for L = 1/2 |m - tgt|^2, evaluated exactly as
    sum (m+ - m-) . ((m+ + m-)/2 - tgt) / (2 eps): the same central difference without
    subtracting two loss values of size ~1e5 (which would cancel)."""
    return float(((mp - mm) * (0.5 * (mp + mm) - tgt)).sum()) / (2 * eps)


@pytest.mark.parametrize("n,k", [((32, 16), 2e-3), ((64, 128), 2e-5)])
def test_adjoint_gradient_matches_oracle(n, k):
    """(32, 16) runs the generic-length kernels, (64, 128) the compile-time-length ones
    (the oracle uses its radix-2 FFT there, pinned against the naive DFT)."""
    if n[0] >= 64:
        O.set_transform(O.FFT)
    try:
        _adjoint_vs_oracle(n, k)
    finally:
        O.set_transform(O.DFT)


def _adjoint_vs_oracle(n, k):
    og = O.Grid(n)
    ctx = L.Context(n)
    m0 = I.smooth2d(n, seed=31, noise=0.05)
    tgt = I.smooth2d(n, seed=32, noise=0.3)
    alpha, h, nsteps = 0.1, (0.1, -0.2, 0.5), 5
    opts = L.Opts(rtol=1e-13, picard_tol=1e-13, restart=30)
    loss, da, dh, dm0 = loss_and_grads(ctx, torch.tensor(m0, device="cuda"), torch.tensor(tgt, device="cuda"),
                                       alpha, h, k, nsteps, opts, checkpoint=2)
    po = O.Params(alpha=alpha, k=k, theta=0.5, lam=0.5, h=h)
    oo = O.Opts(rtol=1e-13, picard_tol=1e-14, picard_max=100)
    lo, da_o, dh_o, dm_o, _ = O.midpoint_loss_grad(og, po, oo, m0, tgt, nsteps)
    assert abs(loss - lo) <= 1e-10 * abs(lo)
    assert abs(da - da_o) <= 1e-8 * abs(da_o)
    assert np.abs(dh - dh_o).max() <= 1e-8 * np.abs(dh_o).max()
    dm = dm0.cpu().numpy()
    assert np.abs(dm - dm_o).max() <= 1e-8 * np.abs(dm_o).max()


@pytest.mark.parametrize("n,k", [((32, 16), 2e-3), ((64, 128), 2e-5)])
def test_adjoint_step_with_nodal_field_matches_oracle(n, k):
    """One converged midpoint step with a per-node applied field h_field: the adjoint's
    mbar_n, d/dalpha (which carries -2 alpha (h + h_field_j) in dR_v/dalpha) and d/dh
    against the oracle's adjoint of the same step, 1e-8 relative.  Both take the step's
    (m^n, v, r) from the oracle's forward, so only the adjoints are compared."""
    if n[0] >= 64:
        O.set_transform(O.FFT)
    try:
        og = O.Grid(n)
        ctx = L.Context(n)
        m0 = I.smooth2d(n, seed=51, noise=0.05)
        mbar = I.smooth2d(n, seed=52, noise=0.3)
        hf = 2.0 * np.random.default_rng(53).standard_normal((3, n[1], n[0]))
        alpha, h = 0.3, (0.1, -0.2, 0.5)
        po = O.Params(alpha=alpha, k=k, theta=0.5, lam=0.5, h=h, h_field=hf)
        oo = O.Opts(rtol=1e-13, picard_tol=1e-14, picard_max=100)
        _, x, _ = O.step_midpoint(og, po, oo, m0)
        mb_o, da_o, dh_o, _ = O.adjoint_midpoint(og, po, oo, m0, x, mbar)
        _, da_0, _, _ = O.adjoint_midpoint(og, O.Params(alpha=alpha, k=k, theta=0.5, lam=0.5, h=h), oo, m0, x, mbar)
        # dropping the field term would miss the 1e-8 comparison below by more than 1000x
        assert abs(da_o - da_0) > 1e3 * 1e-8 * abs(da_o)
        dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")  # noqa: E731
        pl = L.Params(alpha=alpha, k=k, theta=0.5, lam=0.5, h_ext=h, h_field=dev(hf))
        mb, da, dh, info = L.llg_adjoint_step(ctx, pl, L.Opts(rtol=1e-13, restart=30), dev(m0), dev(x), dev(mbar))
        assert info["rel_res_true"] <= 1e-12
        assert abs(da - da_o) <= 1e-8 * abs(da_o), (da, da_o)
        assert np.abs(np.array(dh) - dh_o).max() <= 1e-8 * np.abs(dh_o).max()
        mbh = mb.cpu().numpy()
        assert np.abs(mbh - mb_o).max() <= 1e-8 * np.abs(mb_o).max()
    finally:
        O.set_transform(O.DFT)


def test_adjoint_vs_central_differences_512sq_16_steps():
    """512^2 grid, 16 midpoint steps at dt = 8x the explicit exchange limit, checkpoint every 4
    steps, smooth seeded target: directional derivatives in alpha, h and m0 from the adjoint
    agree with central differences (step 1e-6) to 1e-6 relative."""
    n = (512, 512)
    ctx = L.Context(n)
    alpha, h = 0.1, (0.0, 0.0, 0.5)
    k_ex = 2 * alpha / ((1 + alpha ** 2) * 2 * (np.pi * 512) ** 2)
    k, nsteps = 8 * k_ex, 16
    m0 = torch.tensor(I.smooth2d(n, seed=41), device="cuda")
    tgt = torch.tensor(I.smooth2d(n, seed=42, noise=0.2), device="cuda")
    opts = L.Opts(rtol=1e-13, picard_tol=1e-13, restart=30)
    loss, da, dh, dm0 = loss_and_grads(ctx, m0, tgt, alpha, h, k, nsteps, opts, checkpoint=4)
    eps = 1e-6
    f = lambda a, hh, mm: forward_mT(ctx, mm, a, hh, k, nsteps)  # noqa: E731
    fd_a = central_difference(f(alpha + eps, h, m0), f(alpha - eps, h, m0), tgt, eps)
    assert abs(fd_a - da) <= 1e-6 * abs(da), (fd_a, da)
    # h: a step of 1e-6 moves m(T) (|m| ~ 1) by only ~5e-12 over these 16 short steps, so
    # FP64 rounding of m leaves ~5 digits of m+ - m-, and the node sum against the oscillating
    # m - m_target cancels ~700-fold: the step-1e-6 difference is good to ~1e-5 here.  The
    # map is nearly linear in h over T ~ 5e-6, so step 1e-3 has negligible truncation error
    # and gives the 1e-6 comparison.
    # every component of h: z at both steps, x and y at step 1e-3
    for comp, eps_h, tol in ((2, 1e-6, 1e-4), (2, 1e-3, 1e-6), (0, 1e-3, 1e-6), (1, 1e-3, 1e-6)):
        hp, hm = list(h), list(h)
        hp[comp] += eps_h
        hm[comp] -= eps_h
        fd_h = central_difference(f(alpha, hp, m0), f(alpha, hm, m0), tgt, eps_h)
        assert abs(fd_h - dh[comp]) <= tol * abs(dh[comp]), (comp, eps_h, fd_h, dh[comp])
    d = torch.tensor(I.smooth2d(n, seed=43, noise=1.0), device="cuda")
    fd_m = central_difference(f(alpha, h, m0 + eps * d), f(alpha, h, m0 - eps * d), tgt, eps)
    ad_m = float((dm0 * d).sum())
    assert abs(fd_m - ad_m) <= 1e-6 * abs(ad_m), (fd_m, ad_m)
