"""Temporal convergence on the GPU: the manufactured solution of Sec. 4.2 (64x64 on
(0, 2 pi)^2, T = 0.1, alpha = 0.2, tolerances 1e-10, restart 50) run through the C ABI with
its forcing passed as the per-node applied field each step (Euler at t_{n+1}, midpoint at
t_{n+1/2}).  The errors must equal the paper's printed values to every printed digit (the
oracle reproduces them too, tests/test_oracle_pins.py), in FP64 and with the FP32-flexible
solver, and the final field must match the oracle's to 1e-8.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2607_15290_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2607_15290_b300 as L  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))["temporal_convergence"]
N = (64, 64)


def run_gpu(scheme, k, precision, alpha=0.2, T=0.1):
    ctx = L.Context(N, (2 * np.pi, 2 * np.pi))
    steps = int(round(T / k))
    m0, _ = I.manufactured2d(N, 0.0, alpha)
    m = torch.tensor(m0, device="cuda")
    opts = L.Opts(restart=50, rtol=1e-10, picard_tol=1e-10, precision=precision)
    vprev = None
    for s in range(steps):
        t = s * k
        if scheme == "euler":
            _, f = I.manufactured2d(N, t + k, alpha)
            prm = L.Params(alpha=alpha, k=k, lam=0.5, h_field=torch.tensor(f, device="cuda"))
            m, x, info = L.llg_step_euler(ctx, prm, opts, m)
        else:
            _, f = I.manufactured2d(N, t + 0.5 * k, alpha)
            prm = L.Params(alpha=alpha, k=k, lam=0.5, h_field=torch.tensor(f, device="cuda"))
            m, x, info = L.llg_step_midpoint(ctx, prm, opts, m, vprev)
            vprev = x[:3].contiguous()
        assert info["rel_res_true"] <= 1e-10, info
    torch.cuda.synchronize()
    mh = m.cpu().numpy()
    me, _ = I.manufactured2d(N, steps * k, alpha)
    ctx.close()
    return float(np.mean([np.abs(mh[c] - me[c]).max() for c in range(3)])), mh


def run_oracle(scheme, k, alpha=0.2, T=0.1):
    g = O.Grid(N, (2 * np.pi, 2 * np.pi))
    steps = int(round(T / k))
    m, _ = I.manufactured2d(N, 0.0, alpha)
    opts = O.Opts(restart=50, rtol=1e-10, picard_tol=1e-10)
    vprev = None
    for s in range(steps):
        t = s * k
        if scheme == "euler":
            _, f = I.manufactured2d(N, t + k, alpha)
            m, _, _ = O.step_euler(g, O.Params(alpha=alpha, k=k, theta=1.0, lam=0.5, h_field=f), opts, m)
        else:
            _, f = I.manufactured2d(N, t + 0.5 * k, alpha)
            m, x, _ = O.step_midpoint(g, O.Params(alpha=alpha, k=k, theta=0.5, lam=0.5, h_field=f), opts, m, vprev)
            vprev = x[:3]
    return m


@pytest.mark.parametrize("precision", [L.PREC_FP64, L.PREC_FP32_FLEX], ids=["fp64", "fp32flex"])
@pytest.mark.parametrize("scheme,order", [("euler", 1), ("midpoint", 2)])
def test_manufactured_errors_match_paper(scheme, order, precision):
    errs = []
    for k, val, tol in zip(GOLD["k"], GOLD[scheme]["value"], GOLD[scheme]["tol"]):
        e, _ = run_gpu(scheme, k, precision)
        assert abs(e - val) <= tol, (k, e, val)
        errs.append(e)
    observed = math.log2(errs[0] / errs[1]) / math.log2(GOLD["k"][0] / GOLD["k"][1])
    assert abs(observed - order) <= GOLD["order_tol"], observed


@pytest.mark.parametrize("scheme", ["euler", "midpoint"])
def test_manufactured_field_matches_oracle(scheme):
    O.set_transform(O.FFT)
    try:
        ref = run_oracle(scheme, 1e-2)
    finally:
        O.set_transform(O.DFT)
    _, got = run_gpu(scheme, 1e-2, L.PREC_FP64)
    assert float(np.abs(got - ref).max() / np.abs(ref).max()) <= 1e-8
