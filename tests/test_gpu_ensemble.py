"""Batched ensembles: independent 2D problems of different sizes, damping values and time
steps advanced by projected-Euler steps in one persistent launch, compared problem by
problem with the one-problem-at-a-time context path and with the oracle.

Both paths solve every linear system to a true relative residual of 1e-10, so the
updated fields agree to ~k * 1e-10 |v| (far below 1e-11 here); the comparison uses 1e-10.
"""
import numpy as np
import pytest

import oracle as O
from paper_2607_15290_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2607_15290_b300 as L  # noqa: E402


def k_explicit(alpha, n):
    return 2 * alpha / ((1 + alpha ** 2) * 2 * (np.pi * n) ** 2)


SPECS = [  # (n, alpha, dt / explicit limit, field); rows and columns of different lengths too
    (128, 0.05, 2.0, "smooth"), (128, 0.3, 16.0, "broadband"),
    (256, 0.1, 4.0, "broadband"), (256, 0.4, 8.0, "smooth"),
    (512, 0.02, 3.0, "smooth"), (512, 0.2, 12.0, "broadband"),
    ((512, 128), 0.15, 6.0, "broadband"), ((128, 256), 0.08, 5.0, "smooth"),
]


def shape(n):
    return n if isinstance(n, tuple) else (n, n)


def field(n, kind, seed):
    return I.smooth2d(shape(n), seed=seed) if kind == "smooth" else I.broadband(shape(n), seed=seed)


def test_ensemble_matches_single_problem_path_and_oracle():
    stream = torch.cuda.Stream()
    opts = L.Opts(restart=30, rtol=1e-10, max_iters=600, precision=L.PREC_FP32_FLEX)
    probs, refs, m0s = [], [], []
    for i, (n, alpha, c, kind) in enumerate(SPECS):
        m0 = field(n, kind, 300 + i)
        nn = shape(n)
        prm = L.Params(alpha=alpha, k=c * k_explicit(alpha, max(nn)), lam=0.5, h_ext=(0.0, 0.0, 0.5))
        probs.append({"n": nn, "params": prm, "m": torch.tensor(m0, device="cuda"),
                      "x": torch.zeros((4, nn[1], nn[0]), dtype=torch.float64, device="cuda")})
        m0s.append(m0)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ens = L.Ensemble(probs, opts, stream=stream)
        infos, used_graph = ens.run(2)
    stream.synchronize()
    for i, ((n, alpha, c, kind), p, info) in enumerate(zip(SPECS, probs, infos)):
        assert info["status"] == 0 and info["rel_res_true"] <= 1e-10, (i, info)
        ctx = L.Context(shape(n))
        m = torch.tensor(m0s[i], device="cuda")
        for _ in range(2):
            m, x, _ = L.llg_step_euler(ctx, p["params"], opts, m)
        torch.cuda.synchronize()
        err = float((p["m"] - m).abs().max())
        assert err <= 1e-10, (i, err)
        ctx.close()
    # one problem against the oracle (two Euler steps, 128^2)
    n, alpha, c, kind = SPECS[1]
    g = O.Grid((n, n))
    po = O.Params(alpha=alpha, k=c * k_explicit(alpha, n), lam=0.5, h=(0.0, 0.0, 0.5))
    O.set_transform(O.FFT)
    try:
        mo = m0s[1]
        for _ in range(2):
            mo, _, _ = O.step_euler(g, po, O.Opts(rtol=1e-12, restart=30), mo)
    finally:
        O.set_transform(O.DFT)
    assert np.abs(probs[1]["m"].cpu().numpy() - mo).max() <= 1e-10
    ens.close()
