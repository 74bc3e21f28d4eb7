"""Differentiation through the C ABI: forces as the backward of the energy,
and the hand-written gradient of the energy with respect to the epsilon and
sigma of the inter-molecular term, against central differences of the FP64
oracle's energy (1e-6 relative steps) and of the GPU energy."""
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


def oracle_param_fd(params, pos, types, box, key, k, rel=1e-6):
    p = {q: v.copy() for q, v in params.items()}
    x0 = p[key][k]
    h = rel * x0
    p[key][k] = x0 + h
    ep = Oracle(inputs.params_text(p)).energy(pos, types, box)
    p[key][k] = x0 - h
    em = Oracle(inputs.params_text(p)).energy(pos, types, box)
    return (ep - em) / (2 * h)


@pytest.mark.parametrize("morse", [False, True])
@pytest.mark.parametrize("case", ["hot300", "pe1152"])
def test_param_grad_against_oracle_fd(A, morse, case):
    params = inputs.make_params(0, morse=morse)
    text = inputs.params_text(params)
    if case == "hot300":
        pos, types, box = inputs.amorphous(300, 0.5, 0.9, seed=5)
    else:
        pos, types, box = inputs.polyethylene(3, 4, 8, noise=0.05)
    ev = A.Airebo(text)
    p = torch.tensor(pos, device="cuda")
    ev.neighbor(p, torch.tensor(types, device="cuda"), box)
    _, _, g = ev.param_grad(p)
    eps_key = "morse.epsilon" if morse else "lj.epsilon"
    for k in range(3):
        fd_e = oracle_param_fd(params, pos, types, box, eps_key, k)
        fd_s = oracle_param_fd(params, pos, types, box, "lj.sigma", k)
        assert g[k] == pytest.approx(fd_e, rel=2e-6, abs=1e-6)
        assert g[3 + k] == pytest.approx(fd_s, rel=2e-6, abs=1e-6)


def test_autograd_forces_and_params(A):
    params = inputs.make_params(0)
    text = inputs.params_text(params)
    pos, types, box = inputs.amorphous(300, 0.5, 0.9, seed=5)
    ev = A.Airebo(text)
    p = torch.tensor(pos, device="cuda", requires_grad=True)
    ev.neighbor(p.detach(), torch.tensor(types, device="cuda"), box)
    eps = torch.tensor(params["lj.epsilon"], device="cuda", requires_grad=True)
    sig = torch.tensor(params["lj.sigma"], device="cuda", requires_grad=True)
    E = A.AireboEnergy.apply(p, eps, sig, ev)
    gx, ge, gs = torch.autograd.grad(E, (p, eps, sig))
    f, e4, g = ev.param_grad(p.detach())
    # two evaluations: equal up to the order of FP64 atomic additions
    assert (gx + f).abs().max().item() <= 1e-12 * f.abs().max().item()
    assert np.allclose(ge.cpu().numpy(), g[:3]) and np.allclose(gs.cpu().numpy(), g[3:])
    # central differences of the GPU energy for a few coordinates
    h = 1e-5
    for a in (3, 77, 201):
        for d in range(3):
            q = p.detach().clone(); q[d, a] += h
            ep = ev.compute(q)[1][0].item()
            q[d, a] -= 2 * h
            em = ev.compute(q)[1][0].item()
            assert gx[d, a].item() == pytest.approx((ep - em) / (2 * h), rel=1e-5, abs=1e-7)


def test_fitting_loss_over_64_perturbed_copies(A):
    """A fitting-style loss over 64 perturbed copies of a 2,048-atom amorphous
    C:H box (density 1.0 g/cm^3, H/C = 1): L = sum_c (E_c - E_ref,c)^2 with
    reference energies from shifted parameters; its autograd gradient with
    respect to eps and sigma against central differences of L."""
    params = inputs.make_params(0)
    text = inputs.params_text(params)
    pos0, types, box = inputs.amorphous(2048, 1.0, 1.0, seed=21)
    rng = np.random.default_rng(5)
    copies = [pos0 + rng.normal(0.0, 0.02, pos0.shape) for _ in range(64)]
    ev = A.Airebo(text)
    t = torch.tensor(types, device="cuda")
    ev.neighbor(torch.tensor(pos0, device="cuda"), t, box)
    eps_ref = torch.tensor(params["lj.epsilon"] * 1.05, device="cuda")
    sig_ref = torch.tensor(params["lj.sigma"] * 0.99, device="cuda")
    e_ref = []
    for c in copies:
        e_ref.append(A.AireboEnergy.apply(torch.tensor(c, device="cuda"), eps_ref, sig_ref, ev).item())

    def loss_of(eps, sig, grad):
        total = 0.0
        for c, er in zip(copies, e_ref):
            E = A.AireboEnergy.apply(torch.tensor(c, device="cuda"), eps, sig, ev)
            total = total + (E - er) ** 2
        return total

    eps = torch.tensor(params["lj.epsilon"], device="cuda", requires_grad=True)
    sig = torch.tensor(params["lj.sigma"], device="cuda", requires_grad=True)
    L = loss_of(eps, sig, True)
    ge, gs = torch.autograd.grad(L, (eps, sig))
    for k in (0, 2):
        for which, base, g in (("eps", params["lj.epsilon"], ge), ("sig", params["lj.sigma"], gs)):
            h = 1e-6 * base[k]
            vals = []
            for sgn in (1, -1):
                e = torch.tensor(params["lj.epsilon"], device="cuda")
                s = torch.tensor(params["lj.sigma"], device="cuda")
                (e if which == "eps" else s)[k] += sgn * h
                vals.append(loss_of(e, s, False).item())
            fd = (vals[0] - vals[1]) / (2 * h)
            assert g[k].item() == pytest.approx(fd, rel=1e-4, abs=1e-6)


def test_autograd_knots_and_set_knots(A):
    """The spline knot data as a differentiable input of AireboEnergy: the
    energy after set_knots equals the oracle's with the same knot data, and
    the autograd gradient along a random direction in knot space equals
    central differences of the oracle energy (1e-6 relative step)."""
    params = inputs.make_params(0)
    text = inputs.params_text(params)
    pos, types, box = inputs.amorphous(300, 0.5, 0.9, seed=5)
    ev = A.Airebo(text)
    p = torch.tensor(pos, device="cuda")
    ev.neighbor(p, torch.tensor(types, device="cuda"), box)
    rng = np.random.default_rng(17)
    k0 = A.knot_vector(params)
    # perturbed knot data: the GPU energy follows the oracle's with the same data
    k1 = k0 * (1.0 + 0.05 * rng.uniform(-1, 1, k0.size))
    p1, o = dict(params), 0
    for name, c in A.KNOT_BLOCKS:
        p1[name] = k1[o:o + c].copy()
        o += c
    ev.set_knots(k1)
    e1 = ev.compute(p)[1][0].item()
    want = Oracle(inputs.params_text(p1)).energy(pos, types, box)
    assert e1 == pytest.approx(want, rel=1e-10)
    with pytest.raises(A.AireboError):
        ev.set_knots(k1[:-1])
    # gradient through autograd
    eps = torch.tensor(params["lj.epsilon"], device="cuda")
    sig = torch.tensor(params["lj.sigma"], device="cuda")
    kt = torch.tensor(k0, device="cuda", requires_grad=True)
    E = A.AireboEnergy.apply(p, eps, sig, ev, kt)
    (gk,) = torch.autograd.grad(E, (kt,))
    v = rng.normal(0.0, 1.0, k0.size) * np.maximum(np.abs(k0), 1e-3)
    h = 1e-6
    vals = []
    for sgn in (1, -1):
        q, o = dict(params), 0
        for name, c in A.KNOT_BLOCKS:
            q[name] = k0[o:o + c] + sgn * h * v[o:o + c]
            o += c
        vals.append(Oracle(inputs.params_text(q)).energy(pos, types, box))
    fd = (vals[0] - vals[1]) / (2 * h)
    assert float(gk.cpu().numpy() @ v) == pytest.approx(fd, rel=1e-5, abs=1e-7)


def oracle_force_fd(params, pos, types, box, key, k, rel=1e-6):
    """Central differences of the oracle's forces in one parameter."""
    p = {q: v.copy() for q, v in params.items()}
    x0 = p[key][k]
    h = rel * x0
    p[key][k] = x0 + h
    fp = Oracle(inputs.params_text(p)).compute(pos, types, box)[1]
    p[key][k] = x0 - h
    fm = Oracle(inputs.params_text(p)).compute(pos, types, box)[1]
    return (fp - fm) / (2 * h)


@pytest.mark.parametrize("morse", [False, True])
@pytest.mark.parametrize("case", ["hot300", "pe1152"])
def test_force_param_grad_against_oracle_fd(A, morse, case):
    """v . dF/d(eps, sigma) (the hand-written second derivative of the
    inter-molecular term: radial part, C_ij path, reverse b*) against central
    differences of the oracle's forces with 1e-6 relative steps."""
    params = inputs.make_params(0, morse=morse)
    text = inputs.params_text(params)
    if case == "hot300":
        pos, types, box = inputs.amorphous(300, 0.5, 0.9, seed=5)
    else:
        pos, types, box = inputs.polyethylene(3, 4, 8, noise=0.05)
    v = np.random.default_rng(3).normal(0.0, 1.0, pos.shape)
    ev = A.Airebo(text)
    p = torch.tensor(pos, device="cuda")
    ev.neighbor(p, torch.tensor(types, device="cuda"), box)
    f, _, g = ev.force_param_grad(p, torch.tensor(v, device="cuda"))
    f0, _, _ = ev.compute(p)
    assert (f - f0).abs().max().item() <= 1e-12 * f0.abs().max().item()
    eps_key = "morse.epsilon" if morse else "lj.epsilon"
    for k in range(3):
        for slot, key in ((k, eps_key), (3 + k, "lj.sigma")):
            want = float((v * oracle_force_fd(params, pos, types, box, key, k)).sum())
            assert g[slot] == pytest.approx(want, rel=1e-5, abs=1e-6 * max(1.0, abs(want))), (key, k)


def test_force_param_grad_mixed_close_to_fp64(A, param_text):
    pos, types, box = inputs.amorphous(300, 0.5, 0.9, seed=5)
    v = torch.tensor(np.random.default_rng(4).normal(0.0, 1.0, pos.shape), device="cuda")
    out = []
    for prec in (A.FP64, A.MIXED):
        ev = A.Airebo(param_text, precision=prec)
        p = torch.tensor(pos, device="cuda")
        ev.neighbor(p, torch.tensor(types, device="cuda"), box)
        out.append(ev.force_param_grad(p, v)[2])
    assert np.abs(out[1] - out[0]).max() <= 1e-4 * np.abs(out[0]).max()


def test_force_matching_loss_over_64_perturbed_copies(A):
    """The force-matching loss L = sum_c |F_c - F_ref,c|^2 over 64 perturbed
    copies of a 2,048-atom amorphous C:H box (density 1.0 g/cm^3, H/C = 1),
    F_ref from shifted parameters: its autograd gradient with respect to eps
    and sigma (AireboForces) against central differences of L (1e-5 relative
    steps: the loss sums 64 x 6,144 squared force differences, and the order
    of the FP64 atomic force sums makes each evaluation of L differ at the
    1e-11 level)."""
    params = inputs.make_params(0)
    text = inputs.params_text(params)
    pos0, types, box = inputs.amorphous(2048, 1.0, 1.0, seed=21)
    rng = np.random.default_rng(5)
    copies = [torch.tensor(pos0 + rng.normal(0.0, 0.02, pos0.shape), device="cuda") for _ in range(64)]
    ev = A.Airebo(text)
    ev.neighbor(copies[0], torch.tensor(types, device="cuda"), box)
    eps_ref = torch.tensor(params["lj.epsilon"] * 1.05, device="cuda")
    sig_ref = torch.tensor(params["lj.sigma"] * 0.99, device="cuda")
    f_ref = [A.AireboForces.apply(c, eps_ref, sig_ref, ev).detach() for c in copies]

    def loss_of(eps, sig):
        total = 0.0
        for c, fr in zip(copies, f_ref):
            total = total + ((A.AireboForces.apply(c, eps, sig, ev) - fr) ** 2).sum()
        return total

    eps = torch.tensor(params["lj.epsilon"], device="cuda", requires_grad=True)
    sig = torch.tensor(params["lj.sigma"], device="cuda", requires_grad=True)
    ge, gs = torch.autograd.grad(loss_of(eps, sig), (eps, sig))
    for k in (0, 1, 2):
        for which, base, g in (("eps", params["lj.epsilon"], ge), ("sig", params["lj.sigma"], gs)):
            h = 1e-5 * base[k]
            vals = []
            for sgn in (1, -1):
                e = torch.tensor(params["lj.epsilon"], device="cuda")
                s = torch.tensor(params["lj.sigma"], device="cuda")
                (e if which == "eps" else s)[k] += sgn * h
                vals.append(loss_of(e, s).item())
            fd = (vals[0] - vals[1]) / (2 * h)
            assert g[k].item() == pytest.approx(fd, rel=1e-5), (which, k)
