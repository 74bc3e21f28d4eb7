"""The MD step without host synchronisation (airebo_nve_async) and its CUDA
graph (airebo_graph_capture_nve): the rebuild decision is taken on the
device, and the results equal those of airebo_nve, which decides on the host,
step for step -- positions, velocities, energies and the number of list
builds -- for one system and for a batch of independent systems."""
import numpy as np
import pytest

from paper_1810_07026_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def A():
    from paper_1810_07026_gb300 import build, airebo
    build.build()
    return airebo


def start(A, text, precision, pos, types, box, vel, stream, skin, batch=None):
    ev = A.Airebo(text, precision=precision, skin=skin, stream=stream)
    p = torch.tensor(pos, device="cuda")
    v = torch.tensor(vel, device="cuda")
    t = torch.tensor(types, device="cuda")
    if batch is None:
        ev.neighbor(p, t, box)
    else:
        ev.neighbor_batch(p, t, *batch)
    f, _, _ = ev.compute(p)
    return ev, p, v, f


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_and_async_equal_host_decided_steps(A, param_text, precision):
    prec = A.FP64 if precision == "fp64" else A.MIXED
    pos, types, box = inputs.polyethylene(3, 4, 8, noise=0.03)
    vel = inputs.velocities(types, 600.0, seed=4)
    skin, dt, K, reps = 0.2, 0.5, 10, 3          # a small skin: several rebuilds in 30 steps
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ev, p, v, f = start(A, param_text, prec, pos, types, box, vel, stream, skin)
        for _ in range(K * reps):
            e_ref = ev.nve(p, v, f, dt, 1)
        stream.synchronize()
        x_ref, v_ref, e_ref = p.cpu().numpy(), v.cpu().numpy(), e_ref.cpu().numpy()
        ev.close()
        # the same steps as one captured graph of K steps, launched three times
        ev, p, v, f = start(A, param_text, prec, pos, types, box, vel, stream, skin)
        e4 = ev.graph_capture_nve(p, v, f, dt, K)
        for _ in range(reps):
            ev.graph_launch()
        ev.check()
        stream.synchronize()
        x_g, v_g, e_g = p.cpu().numpy(), v.cpu().numpy(), e4.cpu().numpy()
        ev.close()
        # and directly, without a graph
        ev, p, v, f = start(A, param_text, prec, pos, types, box, vel, stream, skin)
        e4 = ev.nve_async(p, v, f, dt, K * reps)
        ev.check()
        stream.synchronize()
        x_a, e_a = p.cpu().numpy(), e4.cpu().numpy()
        builds = ev.counters()["list_builds"]
        ev.close()
    assert e_ref[3] >= 3, "the test needs rebuilds"
    # the capture rebuilds the lists once at the start (with headroom) before the steps
    assert e_g[3] == e_ref[3] + 1 and e_a[3] == e_ref[3] == builds
    xtol = 1e-9 if precision == "fp64" else 1e-6
    for x in (x_g, x_a):
        assert np.abs(x - x_ref).max() < xtol
    assert np.abs(v_g - v_ref).max() < xtol
    for e in (e_g, e_a):
        assert abs(e[2] - e_ref[2]) <= (1e-10 if precision == "fp64" else 1e-6) * abs(e_ref[2])


def test_batched_graph_md_equals_per_system_steps(A, param_text):
    """Eight amorphous C:H boxes in one handle: ten MD steps in one graph
    launch equal ten steps of each box on its own handle (FP64: the batch
    rebuilds when any box needs it, each handle when its own box does, so the
    order of the sums differs and only FP64 rounding separates the two)."""
    P, T, O, B = inputs.ensemble(8, nmin=200, nmax=800)
    vel = inputs.velocities(T, 300.0, seed=5)
    dt, K = 0.25, 10
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ev, p, v, f = start(A, param_text, A.FP64, P, T, None, vel, stream, 1.0, batch=(O, B))
        ev.graph_capture_nve(p, v, f, dt, K)
        ev.graph_launch()
        ev.check()
        stream.synchronize()
        x_b = p.cpu().numpy()
        ev.close()
        for s in range(len(B)):
            sl = slice(O[s], O[s + 1])
            e2, p2, v2, f2 = start(A, param_text, A.FP64, np.ascontiguousarray(P[:, sl]), T[sl], B[s],
                                   np.ascontiguousarray(vel[:, sl]), stream, 1.0)
            e2.nve(p2, v2, f2, dt, K)
            stream.synchronize()
            assert np.abs(p2.cpu().numpy() - x_b[:, sl]).max() < 1e-9
            e2.close()


def test_async_nonfinite_is_reported_by_check(A, param_text):
    pos, types, box = inputs.diamond()
    vel = inputs.velocities(types, 300.0, seed=1)
    vel[0, 5] = np.nan
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ev, p, v, f = start(A, param_text, A.FP64, pos, types, box, vel, stream, 1.0)
        ev.nve_async(p, v, f, 0.5, 3)
        with pytest.raises(A.AireboError) as ex:
            ev.check()
        assert ex.value.status == A.ERR_NONFINITE
        ev.close()
