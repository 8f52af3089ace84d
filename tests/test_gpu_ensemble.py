"""Batched ensembles: independent 2D problems of different sizes, damping values and time
steps advanced by projected-Euler steps in one persistent launch under a CUDA graph.

* The full batched workload (96 problems: 32 each of 128^2, 256^2 and 512^2, seeded alpha,
  time step and field mix, 5 Euler steps, FP32-flexible GMRES(30) at rtol 1e-10), as
  bench.py runs it: the graph is asserted to have been used; one problem of each size is
  compared with the oracle's five Euler steps (rtol 1e-12) to 1e-10, and every problem with
  the one-problem-at-a-time context path to 1e-10.
* A hand-picked mix that adds rectangular grids, against the context path.

Both GPU paths solve every linear system to a true relative residual of 1e-10, so the
updated fields agree to ~k * 1e-10 |v| (far below 1e-11 here); the comparison uses 1e-10.
The oracle trajectories run in spawned worker processes while the GPU works.
"""
import concurrent.futures as cf
import multiprocessing as mp

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


def make_problem(nn, alpha, k, m0):
    prm = L.Params(alpha=alpha, k=k, lam=0.5, h_ext=(0.0, 0.0, 0.5))
    return {"n": nn, "params": prm, "m": torch.tensor(m0, device="cuda"),
            "x": torch.zeros((4, nn[1], nn[0]), dtype=torch.float64, device="cuda")}


def run_ensemble(probs, opts, steps):
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ens = L.Ensemble(probs, opts, stream=stream)
        infos, used_graph = ens.run(steps)
    stream.synchronize()
    ens.close()
    return infos, used_graph


def against_context_path(probs, m0s, opts, steps):
    ctxs = {}
    for i, p in enumerate(probs):
        nn = p["n"]
        if nn not in ctxs:
            ctxs[nn] = L.Context(nn)
        m = torch.tensor(m0s[i], device="cuda")
        for _ in range(steps):
            m, x, _ = L.llg_step_euler(ctxs[nn], p["params"], opts, m)
        torch.cuda.synchronize()
        err = float((p["m"] - m).abs().max())
        assert err <= 1e-10, (i, nn, err)
    for c in ctxs.values():
        c.close()


def test_full_ensemble_workload_matches_oracle():
    steps = 5
    mix = I.ensemble_mix()
    picks = [next(i for i, s in enumerate(mix) if s[0] == n) for n in (128, 256, 512)]
    oo = O.Opts(rtol=1e-12, restart=30, max_iters=4000)
    pool = cf.ProcessPoolExecutor(max_workers=len(picks), mp_context=mp.get_context("spawn"))
    futs = {}
    for i in picks:
        n, alpha, c, m0 = mix[i]
        po = O.Params(alpha=alpha, k=c * k_explicit(alpha, n), lam=0.5, h=(0.0, 0.0, 0.5))
        futs[i] = pool.submit(O.run_euler, O.Grid((n, n)), po, oo, m0, steps, O.FFT)
    try:
        opts = L.Opts(restart=30, rtol=1e-10, max_iters=900, precision=L.PREC_FP32_FLEX)
        probs = [make_problem((n, n), alpha, c * k_explicit(alpha, n), m0) for n, alpha, c, m0 in mix]
        infos, used_graph = run_ensemble(probs, opts, steps)
        assert used_graph, "the ensemble did not run under its CUDA graph"
        assert len(infos) == len(mix)
        for i, info in enumerate(infos):
            assert info["status"] == 0 and info["rel_res_true"] <= 1e-10, (i, info)
        against_context_path(probs, [s[3] for s in mix], opts, steps)
        for i in picks:
            mo, oinf = futs[i].result()
            assert all(f.converged for f in oinf)
            err = float(np.abs(probs[i]["m"].cpu().numpy() - mo).max())
            assert err <= 1e-10, (i, mix[i][0], err)
    finally:
        pool.shutdown(cancel_futures=True)


def test_ensemble_mixed_shapes_match_single_problem_path():
    opts = L.Opts(restart=30, rtol=1e-10, max_iters=600, precision=L.PREC_FP32_FLEX)
    m0s = [field(n, kind, 300 + i) for i, (n, _, _, kind) in enumerate(SPECS)]
    probs = [make_problem(shape(n), alpha, c * k_explicit(alpha, max(shape(n))), m0)
             for (n, alpha, c, _), m0 in zip(SPECS, m0s)]
    infos, used_graph = run_ensemble(probs, opts, 2)
    assert used_graph
    for i, info in enumerate(infos):
        assert info["status"] == 0 and info["rel_res_true"] <= 1e-10, (i, info)
    against_context_path(probs, m0s, opts, 2)


def test_barrier_wait_limit_returns_timeout_and_ensemble_recovers():
    """The persistent kernel's grid barrier gives up after a clock budget.  With a budget of
    about 1 ms and block 0 withholding its first arrival, every other block's wait runs out:
    the run returns LLG_ERR_TIMEOUT naming the barrier's source line, every block has
    returned (the stream synchronises), and the same ensemble then runs normally and gives
    the context path's result."""
    specs = [(128, 0.1, 4.0, "smooth"), (128, 0.3, 8.0, "broadband")]
    opts = L.Opts(restart=30, rtol=1e-10, max_iters=600, precision=L.PREC_FP32_FLEX)
    m0s = [field(n, kind, 400 + i) for i, (n, _, _, kind) in enumerate(specs)]
    probs = [make_problem(shape(n), alpha, c * k_explicit(alpha, n), m0)
             for (n, alpha, c, _), m0 in zip(specs, m0s)]
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ens = L.Ensemble(probs, opts, stream=stream)
        ens.set_barrier_test(2_000_000, 0)
        with pytest.raises(L.LLGError) as err:
            ens.run(1)
        assert err.value.status == 6, err.value          # LLG_ERR_TIMEOUT
        assert "source line" in str(err.value)
        ens.set_barrier_test(0, -1)
        for p, m0 in zip(probs, m0s):
            p["m"].copy_(torch.tensor(m0, device="cuda"))
        infos, used_graph = ens.run(1)
    stream.synchronize()
    assert used_graph
    for i, info in enumerate(infos):
        assert info["status"] == 0 and info["rel_res_true"] <= 1e-10, (i, info)
    against_context_path(probs, m0s, opts, 1)
    ens.close()
