"""Batched independent systems through the C ABI: every system's energy and
forces equal the oracle's for that system alone; the captured CUDA graph and
the asynchronous evaluation reproduce the synchronous one."""
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


def systems():
    out = [inputs.amorphous(150, 1.0, 1.0, seed=31), inputs.diamond(),
           inputs.amorphous_kd(700, 1.7, 0.9, seed=4), inputs.polyethylene(2, 3, 4, noise=0.05),
           inputs.amorphous_kd(300, 0.6, 0.9, seed=9)]
    pos = np.hstack([s[0] for s in out])
    types = np.concatenate([s[1] for s in out])
    offsets = np.concatenate([[0], np.cumsum([len(s[1]) for s in out])]).astype(np.int64)
    boxes = np.array([s[2] for s in out])
    return out, pos, types, offsets, boxes


@pytest.mark.parametrize("precision,etol,ftol", [(0, 1e-10, 1e-8), (1, 1e-5, 1e-4), (2, 1e-10, 1e-8)])
def test_batched_systems_match_oracle(A, param_text, precision, etol, ftol):
    sysl, pos, types, offsets, boxes = systems()
    ev = A.Airebo(param_text, precision=precision)
    p = torch.tensor(pos, device="cuda")
    ev.neighbor_batch(p, torch.tensor(types, device="cuda"), offsets, boxes)
    f, e = ev.compute_batch(p)
    f, e = f.cpu().numpy(), e.cpu().numpy()
    o = Oracle(param_text)
    for s, (ps, ts, bs) in enumerate(sysl):
        eo, fo, _, _ = o.compute(ps, ts, bs)
        assert abs(e[s] - eo[0]) <= etol * abs(eo[0])
        fs = f[:, offsets[s]:offsets[s + 1]]
        assert np.abs(fs - fo).max() <= ftol * np.abs(fo).max()
    # the total of the per-system energies is the total energy
    _, e4, _ = ev.compute(p)
    assert abs(e.sum() - e4[0].item()) <= 1e-12 * abs(e4[0].item())


@pytest.mark.parametrize("precision", [1, 2])
def test_graph_and_async_reproduce_sync(A, param_text, precision):
    sysl, pos, types, offsets, boxes = systems()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ev = A.Airebo(param_text, precision=precision, stream=stream)
        p = torch.tensor(pos, device="cuda")
        ev.neighbor_batch(p, torch.tensor(types, device="cuda"), offsets, boxes)
        f0, e0 = ev.compute_batch(p)
        f = torch.zeros_like(p)
        e = torch.zeros(len(sysl), dtype=torch.float64, device="cuda")
        ev.graph_capture(p, f, None, e)
        for _ in range(3):
            f.zero_(); e.zero_()
            ev.graph_launch()
            stream.synchronize()
            ev.check()
            assert (f - f0).abs().max().item() <= 1e-12 * f0.abs().max().item()
            assert (e - e0).abs().max().item() <= 1e-12 * e0.abs().max().item()
        f.zero_()
        ev.compute_async(p, f, None, e)
        ev.check()
        assert (f - f0).abs().max().item() <= 1e-12 * f0.abs().max().item()


def test_relaxation_lowers_every_energy(A, param_text):
    from paper_1810_07026_gb300 import batch
    pos, types, offsets, boxes = inputs.ensemble(6, 200, 900, seed=3)
    p = torch.tensor(pos, device="cuda")
    t = torch.tensor(types, device="cuda")
    ev = A.Airebo(param_text)
    ev.neighbor_batch(p, t, offsets, boxes)
    _, e_start = ev.compute_batch(p)
    e_end = batch.relax(param_text, p, t, offsets, boxes, steps=50)
    assert bool((e_end < e_start).all())
