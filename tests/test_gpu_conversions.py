"""The mixed-precision path converts between float and double with integer operations
(the hardware conversions run at the FP64 multiply-add rate on this part) and relies on
them returning exactly the hardware's bits: checked on the device over all 2^32 float
patterns and 2^26 doubles chosen to hit the float range edges, rounding ties and the
subnormal range."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2607_15290_b300 as L  # noqa: E402


def test_integer_conversions_match_hardware():
    ctx = L.Context((8, 8))
    f2d, d2f = ctx.check_conversions(1 << 26)
    assert (f2d, d2f) == (0, 0)
    ctx.close()


def test_check_conversions_rejects_negative_count():
    ctx = L.Context((8, 8))
    with pytest.raises(L.LLGError):
        ctx.check_conversions(-1)
    ctx.close()
