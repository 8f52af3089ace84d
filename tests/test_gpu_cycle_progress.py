"""The two ways the host follows a GMRES cycle give identical results.

By default the Arnoldi kernels publish each cycle's completed step count and stopping flag
in host-mapped memory and the host keeps one step queued; with LLG_HOST_POLL=1 at context
creation (also the path taken where mapped memory is unavailable) it synchronises every
fourth step instead.  The scheduling differs, the arithmetic must not: an FP32-flexible
solve, an all-FP64 solve and two midpoint steps are run both ways, in a child process for
the polling path, and compared bit for bit.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2607_15290_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2607_15290_b300 as L  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N = (32, 32, 32)


def run(out_path):
    """FP32-flexible and FP64 solves and two midpoint steps; arrays saved to out_path."""
    ctx = L.Context(N)
    prm = L.Params(alpha=0.1, k=2e-4, theta=0.5, lam=0.5, h_ext=(0.0, 0.0, 0.5))
    m = torch.tensor(I.smooth3d(N), device="cuda")
    b = L.llg_saddle_apply(ctx, prm, m, torch.tensor(I.random_saddle_vector(N, seed=5), device="cuda"))
    res = {}
    for name, prec in (("flex", L.PREC_FP32_FLEX), ("fp64", L.PREC_FP64)):
        x, info = L.llg_gmres_solve(ctx, prm, L.Opts(restart=30, rtol=1e-11, precision=prec), m, b)
        res[name] = x.cpu().numpy()
        res[name + "_iters"] = np.array([info["iters"], info["restarts"]])
    opts = L.Opts(restart=30, rtol=1e-10, picard_tol=1e-10, precision=L.PREC_FP32_FLEX)
    mm, vprev = m, None
    for s in range(2):
        mm, x, info = L.llg_step_midpoint(ctx, prm, opts, mm, vprev)
        vprev = x[:3].contiguous()
    res["m2"] = mm.cpu().numpy()
    res["m2_iters"] = np.array([info["iters"], info["picard_iters"]])
    ctx.close()
    np.savez(out_path, **res)


def test_mapped_progress_and_polling_agree(tmp_path):
    mapped = tmp_path / "mapped.npz"
    polled = tmp_path / "polled.npz"
    run(str(mapped))
    env = dict(os.environ, LLG_HOST_POLL="1")
    code = ("import sys; sys.path.insert(0, %r); sys.path.insert(0, %r); "
            "import test_gpu_cycle_progress as t; t.run(%r)") % (ROOT, os.path.join(ROOT, "tests"), str(polled))
    subprocess.run([sys.executable, "-c", code], env=env, check=True, cwd=ROOT, timeout=600)
    a, b = np.load(mapped), np.load(polled)
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
