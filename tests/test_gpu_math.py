"""The FP64 reciprocal and reciprocal square root of the kernels (the
hardware approximation refined by one third-order Newton-Raphson step)
against CUDA's correctly rounded results on the device."""
import pytest

pytestmark = pytest.mark.gpu


def test_rcp_rsqrt_within_two_ulp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_07026_gb300 import build, airebo
    build.build()
    ulp_rcp, ulp_rsqrt, raw_rcp, raw_rsqrt = airebo.math_check()
    print(f"ulp: 1/x {ulp_rcp}, 1/sqrt(x) {ulp_rsqrt}; hardware approximations alone {raw_rcp}, {raw_rsqrt}")
    assert ulp_rcp <= 1, ulp_rcp          # faithful: at most one rounding step from 1/x
    assert ulp_rsqrt <= 2, ulp_rsqrt      # the reference 1/sqrt(x) is itself within 1 ulp


def test_double_float_operations():
    """The double-float operations of the DF64 torsion kernel against FP64 on
    the same exactly representable inputs: about 48-bit arithmetic."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_07026_gb300 import build, airebo
    build.build()
    e = airebo.dd_check()
    print(e)
    assert e["add"] <= 2.0 ** -45, e            # relative to |a| + |b|
    for k in ("mul", "div", "rcp", "rsqrt"):
        assert e[k] <= 2.0 ** -44, (k, e)
    assert e["sinpi"] <= 2.0 ** -45 and e["cospi"] <= 2.0 ** -45, e
    assert e["from_double"] <= 2.0 ** -47, e
