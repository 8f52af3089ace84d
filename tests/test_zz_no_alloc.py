"""The allocation-free preconditioner call, llg_ffthss_apply_noalloc.

Some callers cannot allocate device memory (a loop that promised no allocation
after start-up, memory fully reserved by another allocator, a plug-in that may
not create allocations) and so cannot create a context.  This call serves them
from a static device array.  Here it is called through the C ABI twice in a row
(two different grids, so the shared scratch is reused) and each output is
compared with the context entry point llg_ffthss_apply at the FP64 apply
tolerance used elsewhere (1e-12, max-norm relative).  A grid larger than the
stated maximum must be refused before any launch.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2607_15290_b300 as L  # noqa: E402
from paper_2607_15290_b300 import _abi  # noqa: E402
from paper_2607_15290_b300 import inputs as I  # noqa: E402


def _grid(n, Lc):
    g = _abi.Grid()
    g.dim = len(n)
    for i in range(3):
        g.n[i] = n[i] if i < len(n) else 1
        g.L[i] = Lc[i] if i < len(n) else 1.0
    return g


def _noalloc(n, Lc, prm, m, p, transpose):
    z = torch.full_like(p, float("nan"))
    st = _abi.lib().llg_ffthss_apply_noalloc(
        C.byref(_grid(n, Lc)), C.byref(prm.c()), C.c_void_p(m.data_ptr()), C.c_void_p(p.data_ptr()),
        C.c_void_p(z.data_ptr()), int(transpose), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, _abi.STATUS.get(st, st)
    return z


def test_noalloc_matches_context_apply_on_two_calls_in_a_row():
    assert torch.cuda.is_available()
    cases = [
        ((64, 32), (1.0, 2.0), L.Params(alpha=0.1, k=3e-3, theta=1.0, lam=0.5), False, 201),
        ((16, 8, 32), (1.0, 1.0, 0.5), L.Params(alpha=0.2, k=1e-3, theta=0.5, lam=0.25, exchange=L.EX_FD2),
         True, 202),
    ]
    inputs = []
    for n, Lc, prm, tr, seed in cases:
        m = torch.tensor(I.random_unit(n, seed=seed), device="cuda")
        p = torch.tensor(I.random_saddle_vector(n, seed=seed + 1), device="cuda")
        inputs.append((m, p))
    # the two allocation-free calls, back to back on the same stream
    outs = [_noalloc(n, Lc, prm, m, p, tr) for (n, Lc, prm, tr, _), (m, p) in zip(cases, inputs)]
    torch.cuda.synchronize()
    for (n, Lc, prm, tr, _), (m, p), z in zip(cases, inputs, outs):
        ctx = L.Context(n, Lc)
        ref = L.llg_ffthss_apply(ctx, prm, m, p, transpose=tr)
        torch.cuda.synchronize()
        err = float((z - ref).abs().max() / ref.abs().max())
        assert np.isfinite(err) and err <= 1e-12, (n, err)
        ctx.close()


# near the size limit (n1 * n2 * S up to LLG_NOALLOC_MAX_SPECTRAL = 262144), lines of up to
# 1024 points in every axis position, both transpose modes: these FP64 row and column kernels
# run only through this entry point (the context path takes compile-time-length kernels there)
LARGE = [((512, 256), (1.0, 1.0)), ((1024, 128), (1.0, 0.5)), ((2, 1024), (0.25, 1.0)),
         ((64, 64, 32), (1.0, 1.0, 2.0))]


@pytest.mark.parametrize("n,Lc", LARGE, ids=["512x256", "1024x128", "2x1024", "64x64x32"])
@pytest.mark.parametrize("transpose", [False, True], ids=["M", "MT"])
def test_noalloc_matches_context_apply_near_the_size_limit(n, Lc, transpose):
    prm = L.Params(alpha=0.15, k=2e-4, theta=0.5, lam=0.5)
    m = torch.tensor(I.random_unit(n, seed=211), device="cuda")
    p = torch.tensor(I.random_saddle_vector(n, seed=212), device="cuda")
    z = _noalloc(n, Lc, prm, m, p, transpose)
    ctx = L.Context(n, Lc)
    ref = L.llg_ffthss_apply(ctx, prm, m, p, transpose=transpose)
    torch.cuda.synchronize()
    err = float((z - ref).abs().max() / ref.abs().max())
    assert np.isfinite(err) and err <= 1e-12, (n, transpose, err)
    ctx.close()


def test_noalloc_refuses_grids_beyond_its_static_scratch():
    n = (1024, 1024)                       # needs 1024 * 1552 slots > LLG_NOALLOC_MAX_SPECTRAL
    prm = L.Params()
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    ptr = C.c_void_p(dummy.data_ptr())
    st = _abi.lib().llg_ffthss_apply_noalloc(C.byref(_grid(n, (1.0, 1.0))), C.byref(prm.c()), ptr, ptr, ptr, 0,
                                             None)
    assert st == 2   # LLG_ERR_UNSUPPORTED_SIZE, returned before any launch
