"""Launch-shape autotuner: the tuned shapes stay inside the candidate sets and
leave the result unchanged up to the order of floating-point atomic sums."""
import numpy as np
import pytest

from paper_1810_07026_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_autotune_keeps_result(torch_cuda, param_text, prec):
    torch = torch_cuda
    from paper_1810_07026_gb300 import airebo as A
    p = A.FP64 if prec == "fp64" else A.MIXED
    pos0, types, box = inputs.polyethylene(5, 6, 4, seed=3)
    ev = A.Airebo(param_text, precision=p)
    pos = torch.tensor(pos0, device="cuda")
    ev.neighbor(pos, torch.tensor(types, device="cuda"), box)
    f0, e0, _ = ev.compute(pos)
    chunk, grid, bgrid = ev.autotune(pos)
    assert chunk in (2, 4, 8, 16) and grid in (2, 4, 8, 16, 32) and bgrid in (2, 4, 8, 16, 32)
    f1, e1, _ = ev.compute(pos)
    # any launch shape in range gives the same result
    for c, g, b in ((1, 1, 1), (3, 5, 7), (64, 32, 32)):
        ev.set_launch_shape(c, g, b)
        f2, e2, _ = ev.compute(pos)
        assert np.allclose(e2.cpu().numpy(), e0.cpu().numpy(), rtol=1e-12, atol=1e-9)
        assert (f2 - f0).abs().max().item() < 1e-9
    assert np.allclose(e1.cpu().numpy(), e0.cpu().numpy(), rtol=1e-12, atol=1e-9)
    assert (f1 - f0).abs().max().item() < 1e-9
    with pytest.raises(RuntimeError):
        ev.set_launch_shape(0, 8, 8)
    with pytest.raises(RuntimeError):
        ev.set_launch_shape(8, 33, 8)
    with pytest.raises(RuntimeError):
        ev.set_launch_shape(8, 8, 0)
    ev.close()
