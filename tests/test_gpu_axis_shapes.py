"""Axis-pass launch shapes set by hand (llg_set_axis_shape): every shape the tuner would try
gives the FP32 apply of the default shapes (2e-5 against the oracle, as in test_gpu_parity);
shapes the grid does not have are refused."""
import numpy as np
import pytest

import oracle as O
from paper_2607_15290_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2607_15290_b300 as L  # noqa: E402


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.mark.parametrize("n,shapes", [
    ((128, 128, 128), {"y-forward": "register(E8,TW16)", "z": "tma(TW8)", "y-inverse": "register(E8,TW16)"}),
    ((128, 128, 128), {"y-forward": "tma(TW16)", "z": "paired(E8,TW16)", "y-inverse": "staged(TW16,CB8)"}),
    ((128, 128, 128), {"z": "staged(TW32,CB16)"}),
    ((128, 128, 128), {"y-forward": "tma(E16,TW8)", "z": "tma(E16,TW16)", "y-inverse": "tma(E16,TW16)"}),
    ((64, 256, 256), {"y-forward": "tma(E16,TW16)", "z": "tma(E16,TW8)", "y-inverse": "tma(E16,TW8)"}),
], ids=["live-128", "mixed", "z-only", "radix16-128", "radix16-256"])
def test_fixed_shapes_match_oracle(n, shapes):
    og = O.Grid(n)
    ctx = L.Context(n)
    for slot, shape in shapes.items():
        ctx.set_axis_shape(slot, shape)
    m = I.random_unit(n, seed=141)
    p = I.random_saddle_vector(n, seed=142)
    po = O.Params(alpha=0.1, k=1e-6, theta=0.5, lam=0.5)
    pl = L.Params(alpha=0.1, k=1e-6, theta=0.5, lam=0.5)
    O.set_transform(O.FFT)
    try:
        ref = O.ffthss_apply(og, po, m, p)
    finally:
        O.set_transform(O.DFT)
    got = L.llg_ffthss_apply_f32(ctx, pl, torch.tensor(m, dtype=torch.float32, device="cuda"),
                                 torch.tensor(p, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert rel(got.cpu().numpy(), ref) <= 2e-5
    ctx.close()


def test_refused_shapes():
    ctx = L.Context((64, 64))
    with pytest.raises(L.LLGError):
        ctx.set_axis_shape("z", "register(E8,TW8)")       # a 2D grid has no z pass
    with pytest.raises(L.LLGError):
        ctx.set_axis_shape("y(2D)", "register(E8,TW32)")  # no 32-column register tile
    ctx.set_axis_shape("y(2D)", "register(E8,TW8)")
    ctx.close()
