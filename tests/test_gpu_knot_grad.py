"""Gradient of the energy with respect to the spline knot data (the fitting
gradient of the bond-order splines) through the C ABI, against central
differences of the FP64 oracle's energy: along random directions over every
block of knot data, and component by component for the largest entries."""
import numpy as np
import pytest

from paper_1810_07026_gb300 import inputs
from oracle.oracle import Oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def A():
    from paper_1810_07026_gb300 import build, airebo
    build.build()
    return airebo


def split(A, g):
    out, o = {}, 0
    for name, c in A.KNOT_BLOCKS:
        out[name] = g[o:o + c]
        o += c
    return out


def oracle_fd(params, pos, types, box, direction, h):
    """(E(d + h v) - E(d - h v)) / 2h with v given per block."""
    ep = dict(params)
    em = dict(params)
    for k, v in direction.items():
        ep[k] = params[k] + h * v
        em[k] = params[k] - h * v
    e_p = Oracle(inputs.params_text(ep)).energy(pos, types, box)
    e_m = Oracle(inputs.params_text(em)).energy(pos, types, box)
    return (e_p - e_m) / (2 * h)


@pytest.fixture(scope="module")
def case(A):
    params = inputs.make_params(0)
    text = inputs.params_text(params)
    # amorphous C:H (H/C = 1): bond orders visit many spline cells
    pos, types, box = inputs.amorphous(600, 1.0, 1.0, seed=11)
    ev = A.Airebo(text)
    p = torch.tensor(pos, device="cuda")
    ev.neighbor(p, torch.tensor(types, device="cuda"), box)
    f, e4, g = ev.knot_grad(p)
    f0, e0, _ = ev.compute(p)
    ev.close()
    return params, pos, types, box, g, f, e4, f0, e0


def test_knot_grad_keeps_forces_and_energy(A, case):
    params, pos, types, box, g, f, e4, f0, e0 = case
    assert g.shape == (A.KNOT_COUNT,) and np.all(np.isfinite(g))
    assert (f - f0).abs().max().item() <= 1e-12 * f0.abs().max().item()
    assert np.allclose(e4.cpu().numpy(), e0.cpu().numpy(), rtol=1e-12, atol=1e-9)
    blocks = split(A, g)
    # every block is read by some bond order of this system
    for name, v in blocks.items():
        assert np.abs(v).max() > 0, name


BLOCKS = ["gC1.data", "gC2.data", "gH.data", "P.CC", "P.CH", "P.HC", "piRC.CC", "piRC.CH", "piRC.HH", "Tij.CC"]


@pytest.mark.parametrize("block", BLOCKS)
def test_knot_grad_directional_per_block(A, case, block):
    params, pos, types, box, g, *_ = case
    blocks = split(A, g)
    rng = np.random.default_rng(100 + BLOCKS.index(block))
    v = rng.standard_normal(params[block].shape)
    h = 1e-6 * max(1.0, float(np.abs(params[block]).max()))
    fd = oracle_fd(params, pos, types, box, {block: v}, h)
    an = float(blocks[block] @ v)
    assert an == pytest.approx(fd, rel=2e-6, abs=1e-6)


def test_knot_grad_all_blocks_and_largest_components(A, case):
    params, pos, types, box, g, *_ = case
    blocks = split(A, g)
    rng = np.random.default_rng(5)
    v = {k: rng.standard_normal(params[k].shape) * max(1e-2, float(np.abs(params[k]).max()))
         for k, _ in A.KNOT_BLOCKS}
    fd = oracle_fd(params, pos, types, box, v, 1e-6)
    an = sum(float(blocks[k] @ v[k]) for k in v)
    assert an == pytest.approx(fd, rel=2e-6, abs=1e-6)
    # the three largest single entries
    for idx in np.argsort(-np.abs(g))[:3]:
        o = 0
        for name, c in A.KNOT_BLOCKS:
            if idx < o + c:
                e = np.zeros(c)
                e[idx - o] = 1.0
                fd1 = oracle_fd(params, pos, types, box, {name: e}, 1e-5)
                assert g[idx] == pytest.approx(fd1, rel=2e-6, abs=1e-6), (name, idx - o)
                break
            o += c


def test_knot_grad_same_in_df64(A, case):
    """The knots enter only through bond orders, which run in FP64 in both
    precisions: DF64's gradient equals FP64's up to summation order."""
    params, pos, types, box, g, *_ = case
    ev = A.Airebo(inputs.params_text(params), precision=A.DF64)
    p = torch.tensor(pos, device="cuda")
    ev.neighbor(p, torch.tensor(types, device="cuda"), box)
    _, _, g2 = ev.knot_grad(p)
    ev.close()
    assert np.abs(g2 - g).max() <= 1e-10 * np.abs(g).max()


def test_knot_grad_count_checked(A, case):
    params, pos, types, box, *_ = case
    ev = A.Airebo(inputs.params_text(params))
    p = torch.tensor(pos, device="cuda")
    ev.neighbor(p, torch.tensor(types, device="cuda"), box)
    f = torch.empty_like(p)
    e4 = torch.empty(4, dtype=torch.float64, device="cuda")
    g = np.zeros(A.KNOT_COUNT - 1)
    st = A.lib().airebo_knot_grad(ev._h, A._ptr(p), A._ptr(f), A._ptr(e4), A._np(g), A.KNOT_COUNT - 1)
    assert st == 1            # AIREBO_ERR_ARG
    ev.close()
