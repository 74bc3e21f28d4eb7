"""Pins of the CPU oracle against mathematics it must satisfy (no GPU).

* forces equal central finite differences of the energy (all terms together
  and one term at a time);
* translation, rotation and permutation invariance, zero net force;
* the virial equals minus the strain derivative of the energy;
* splines reproduce their knot data (values and derivatives), are C^1 across
  cell faces, clamp outside their domain, and the same-species pi^rc and T
  tables are symmetric in their first two arguments;
* neighbour sets equal a brute-force search over all periodic images;
* the nested-loop C_ij search equals a brute-force enumeration of simple paths;
* velocity-Verlet energy fluctuations shrink as dt^2.
"""
import itertools
import math

import numpy as np
import pytest

from paper_1810_07026_gb300 import inputs
from oracle.oracle import FLAG_REBO, FLAG_LJ, FLAG_TORSION, FLAG_ALL


@pytest.fixture(scope="module")
def hot():
    """A small, non-equilibrated amorphous C:H box: many bonds sit inside
    their switch, many pairs need b*, C_ij takes fractional values."""
    return inputs.amorphous(160, 1.0, 1.0, seed=11, min_sep=1.0)


def fd_forces(oracle, pos, types, box, atoms, flags, h=1e-5):
    out = np.zeros((3, len(atoms)))
    for n, a in enumerate(atoms):
        for d in range(3):
            p = pos.copy(); p[d, a] += h
            ep = oracle.energy(p, types, box, flags)
            p[d, a] -= 2 * h
            em = oracle.energy(p, types, box, flags)
            out[d, n] = -(ep - em) / (2 * h)
    return out


@pytest.mark.parametrize("flags", [FLAG_ALL, FLAG_REBO, FLAG_LJ, FLAG_TORSION])
def test_forces_are_energy_gradient_hot(oracle, hot, flags):
    pos, types, box = hot
    _, f, _, _ = oracle.compute(pos, types, box, flags)
    atoms = list(range(0, 160, 9))
    fd = fd_forces(oracle, pos, types, box, atoms, flags)
    scale = np.abs(f).max()
    assert scale > 0
    assert np.abs(fd - f[:, atoms]).max() <= 2e-6 * scale + 1e-9


def test_forces_are_energy_gradient_diamond_pe(oracle):
    for pos, types, box in (inputs.diamond(), inputs.polyethylene(2, 2, 4, noise=0.05)):
        _, f, _, _ = oracle.compute(pos, types, box)
        atoms = [0, 7, 31, 77]
        fd = fd_forces(oracle, pos, types, box, atoms, FLAG_ALL)
        assert np.abs(fd - f[:, atoms]).max() <= 1e-6 * np.abs(f).max()


def test_hot_system_exercises_branches(oracle, hot):
    pos, types, box = hot
    _, _, _, c = oracle.compute(pos, types, box)
    assert c["bstar"] > 0 and c["bstar_dsb_nonzero"] > 0
    assert c["dihedral_pairs"] > 0 and c["torsion_quads"] > 0
    assert c["lj_c_zero"] > 0


def test_zero_net_force_and_translation(oracle, hot):
    pos, types, box = hot
    e, f, w, _ = oracle.compute(pos, types, box)
    assert np.abs(f.sum(axis=1)).max() < 1e-9 * np.abs(f).max() * len(types)
    shift = np.array([[0.31], [-1.7], [2.2]])
    e2, f2, w2, _ = oracle.compute(pos + shift, types, box)
    assert e2[0] == pytest.approx(e[0], rel=1e-11)
    assert np.abs(f2 - f).max() < 1e-9 * np.abs(f).max()
    assert np.abs(w2 - w).max() < 1e-8 * np.abs(w).max()


def test_permutation_invariance(oracle, hot):
    """b_ij = b_ji: the energy does not depend on which atom of a pair is i."""
    pos, types, box = hot
    e, f, _, _ = oracle.compute(pos, types, box)
    perm = np.random.default_rng(5).permutation(len(types))
    e2, f2, _, _ = oracle.compute(pos[:, perm], types[perm], box)
    assert e2[0] == pytest.approx(e[0], rel=1e-11)
    assert np.abs(f2 - f[:, perm]).max() < 1e-9 * np.abs(f).max()


def cluster():
    pos, types, _ = inputs.amorphous(60, 1.0, 1.0, seed=4)
    return pos + 15.0, types, np.array([45.0, 45.0, 45.0])


def test_rotation_invariance(oracle):
    pos, types, box = cluster()
    e, f, _, _ = oracle.compute(pos, types, box)
    a, b, c = 0.3, -1.1, 2.0
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Ry = np.array([[math.cos(b), 0, math.sin(b)], [0, 1, 0], [-math.sin(b), 0, math.cos(b)]])
    Rx = np.array([[1, 0, 0], [0, math.cos(c), -math.sin(c)], [0, math.sin(c), math.cos(c)]])
    R = Rz @ Ry @ Rx
    ctr = pos.mean(axis=1, keepdims=True)
    pr = R @ (pos - ctr) + ctr
    e2, f2, _, _ = oracle.compute(pr, types, box)
    assert e2[0] == pytest.approx(e[0], rel=1e-11)
    assert np.abs(f2 - R @ f).max() < 1e-9 * np.abs(f).max()


def test_virial_diagonal_is_strain_derivative(oracle, hot):
    pos, types, box = hot
    _, _, w, _ = oracle.compute(pos, types, box)
    h = 1e-6
    for d in range(3):
        s = np.ones(3); s[d] += h
        ep = oracle.energy(pos * s[:, None], types, box * s)
        s[d] -= 2 * h
        em = oracle.energy(pos * s[:, None], types, box * s)
        assert w[d] == pytest.approx(-(ep - em) / (2 * h), rel=1e-6, abs=1e-6)


def test_virial_offdiagonal_is_shear_derivative(oracle):
    pos, types, box = cluster()
    _, _, w, _ = oracle.compute(pos, types, box)
    h = 1e-6
    for k, (a, b) in zip((3, 4, 5), ((0, 1), (0, 2), (1, 2))):
        def e_at(eps):
            p = pos.copy()
            p[a] = pos[a] + eps * pos[b]
            return oracle.energy(p, types, box)
        assert w[k] == pytest.approx(-(e_at(h) - e_at(-h)) / (2 * h), rel=1e-6, abs=1e-6)


# ----------------------------------------------------------------- splines

def test_quintic_knots(oracle, params):
    for which, name in ((0, "gC1"), (1, "gC2"), (2, "gH")):
        kn = params[f"{name}.knots"]
        d = params[f"{name}.data"].reshape(-1, 3)
        for k, c in enumerate(kn):
            v, g = oracle.spline(which, c)
            assert v == pytest.approx(d[k, 0], rel=1e-13)
            assert g[0] == pytest.approx(d[k, 1], rel=1e-10)
            if 0 < k < len(kn) - 1:
                # second derivative from both sides equals the knot datum
                h = 1e-7
                gl = oracle.spline(which, c - h)[1][0]
                gr = oracle.spline(which, c + h)[1][0]
                assert (gr - gl) / (2 * h) == pytest.approx(d[k, 2], rel=1e-5)
        xs = np.linspace(-1, 1, 2001)
        assert min(oracle.spline(which, x)[0] for x in xs) > 0.0


def test_bicubic_knots_and_continuity(oracle, params):
    for which, name in ((10, "CC"), (11, "CH"), (12, "HC")):
        d = params[f"P.{name}"].reshape(5, 5, 4)
        for x in range(5):
            for y in range(5):
                v, g = oracle.spline(which, x, y)
                assert v == pytest.approx(d[x, y, 0], abs=1e-14)
                assert g[0] == pytest.approx(d[x, y, 1], abs=1e-13)
                assert g[1] == pytest.approx(d[x, y, 2], abs=1e-13)
        # C^1 across the face x = 2 at a non-knot y
        e = 1e-9
        vl, gl = oracle.spline(which, 2 - e, 1.37)
        vr, gr = oracle.spline(which, 2 + e, 1.37)
        assert vl == pytest.approx(vr, abs=1e-8)
        assert np.abs(gl - gr).max() < 1e-7
        # clamped outside [0, 4]
        v5, g5 = oracle.spline(which, 5.5, 1.2)
        v4, _ = oracle.spline(which, 4.0, 1.2)
        assert v5 == v4 and g5[0] == 0.0


def test_tricubic_knots_symmetry(oracle, params):
    rng = np.random.default_rng(0)
    for which, name, sym in ((20, "piRC.CC", True), (21, "piRC.CH", False), (22, "piRC.HH", True),
                             (30, "Tij.CC", True)):
        d = params[name].reshape(5, 5, 9, 8)
        for _ in range(20):
            x, y, z = rng.integers(0, 5), rng.integers(0, 5), rng.integers(1, 10)
            v, g = oracle.spline(which, x, y, z)
            assert v == pytest.approx(d[x, y, z - 1, 0], abs=1e-14)
            assert np.abs(g - d[x, y, z - 1, 1:4]).max() < 1e-13
        # cross derivative f_xy at a knot from finite differences of f_x
        h = 1e-7
        gxp = oracle.spline(which, 2, 1 + h, 3)[1][0]
        gxm = oracle.spline(which, 2, 1 - h, 3)[1][0]
        assert (gxp - gxm) / (2 * h) == pytest.approx(d[2, 1, 2, 4], abs=1e-8)
        if sym:
            for _ in range(20):
                a, b, c = rng.uniform(0, 4), rng.uniform(0, 4), rng.uniform(1, 9)
                assert oracle.spline(which, a, b, c)[0] == pytest.approx(oracle.spline(which, b, a, c)[0], abs=1e-14)
        e = 1e-9
        vl, gl = oracle.spline(which, 1.3, 2.6, 4 - e)
        vr, gr = oracle.spline(which, 1.3, 2.6, 4 + e)
        assert vl == pytest.approx(vr, abs=1e-8) and np.abs(gl - gr).max() < 1e-7


def test_switches(oracle):
    for t, v in ((-0.5, 1.0), (0.0, 1.0), (0.5, 0.5), (1.0, 0.0), (2.0, 0.0)):
        assert oracle.spline(40, t)[0] == pytest.approx(v, abs=1e-15)
    assert oracle.spline(40, 0.25)[1][0] == pytest.approx(-0.5 * math.pi * math.sin(math.pi * 0.25))
    assert oracle.spline(41, 0.5)[0] == pytest.approx(0.5)
    assert oracle.spline(41, 0.3)[1][0] == pytest.approx(-6 * 0.3 + 6 * 0.09)


# ------------------------------------------------------ neighbours and C_ij

def brute_pairs(pos, types, box, cut):
    """All (i, j, S) with |x_j + S L - x_i| < cut(t_i, t_j), every image tried."""
    n = len(types)
    out = set()
    rng = [int(math.ceil(cut(0, 0) / L)) + 1 for L in box]
    rc = np.array([[cut(a, b) for b in (0, 1)] for a in (0, 1)])[types[:, None], types[None, :]]
    for S in itertools.product(*(range(-r, r + 1) for r in rng)):
        d = pos[:, None, :] + (np.array(S) * box)[:, None, None] - pos[:, :, None]
        r2 = np.einsum("dij,dij->ij", d, d)
        hit = r2 < rc * rc
        if S == (0, 0, 0):
            np.fill_diagonal(hit, False)
        for i, j in zip(*np.nonzero(hit)):
            out.add((int(i), int(j), S))
    return out


def as_set(off, j, img):
    return {(i, int(j[k]), tuple(int(s) for s in img[k])) for i in range(len(off) - 1) for k in range(off[i], off[i + 1])}


def test_rebo_neighbours_brute_force(oracle, params):
    dmax = params["Dmax"]
    for pos, types, box in (inputs.amorphous(120, 1.0, 1.0, seed=2), inputs.diamond()):
        got = as_set(*oracle.rebo_neighbors(pos, types, box))
        want = brute_pairs(pos, types, box, lambda a, b: dmax[a + b])
        assert got == want


def test_lj_half_pairs_brute_force(oracle, params):
    sig = params["lj.sigma"]
    pos, types, box = inputs.diamond()
    got = as_set(*oracle.lj_pairs(pos, types, box))
    full = brute_pairs(pos, types, box, lambda a, b: 3.0 * sig[a + b])
    want = {(i, j, S) for (i, j, S) in full if j > i or (j == i and S > (0, 0, 0))}
    assert got == want


def test_cij_brute_force_paths(oracle, params, hot):
    """Max over all simple paths of <= 3 bonds, enumerated independently."""
    pos, types, box = hot
    off, jj, img = oracle.rebo_neighbors(pos, types, box)
    nb = [[(int(jj[k]), tuple(int(s) for s in img[k])) for k in range(off[i], off[i + 1])] for i in range(len(types))]
    dmin, dmax = params["Dmin"], params["Dmax"]

    def wgt(a, Sa, b, Sb):
        d = pos[:, b] + np.array(Sb) * box - pos[:, a] - np.array(Sa) * box
        r = math.sqrt(d @ d)
        t = (r - dmin[types[a] + types[b]]) / (dmax[types[a] + types[b]] - dmin[types[a] + types[b]])
        return 1.0 if t <= 0 else 0.0 if t >= 1 else 0.5 * (1 + math.cos(math.pi * t))

    add = lambda A, B: tuple(x + y for x, y in zip(A, B))
    best = {}
    for i in range(len(types)):
        O = (0, 0, 0)
        stack = [((i, O),)]
        while stack:
            path = stack.pop()
            a, Sa = path[-1]
            for b, Sb in nb[a]:
                node = (b, add(Sa, Sb))
                if node in path:
                    continue
                np_ = path + (node,)
                wt = 1.0
                for u, v in zip(np_[:-1], np_[1:]):
                    wt *= wgt(u[0], u[1], v[0], v[1])
                key = (i,) + node
                best[key] = max(best.get(key, 0.0), wt)
                if len(np_) < 4:
                    stack.append(np_)
    checked = 0
    for (i, j, S), wmax in best.items():
        if j == i:
            continue
        c, _ = oracle.cij(i, j, list(S))
        assert c == pytest.approx(1.0 - wmax, abs=1e-14)
        checked += 1
    assert checked > 500
    assert any(0.0 < 1 - v < 1.0 for v in best.values())


# ------------------------------------------------------------------- NVE

def nve_energy_spread(oracle, pos, types, box, vel, dt, t_total):
    m = inputs.masses(types)
    ftoa = 1.0 / inputs.MVV2E
    e, f, _, _ = oracle.compute(pos, types, box)
    x, v = pos.copy(), vel.copy()
    tot = []
    for _ in range(int(round(t_total / dt))):
        v += 0.5 * dt * f / m * ftoa
        x += dt * v
        e, f, _, _ = oracle.compute(x, types, box)
        v += 0.5 * dt * f / m * ftoa
        tot.append(e[0] + 0.5 * inputs.MVV2E * (m * v * v).sum())
    tot = np.array(tot)
    return tot.max() - tot.min(), tot


def test_nve_energy_conservation_dt2(oracle):
    pos, types, box = inputs.diamond()
    vel = inputs.velocities(types, 1000.0, seed=3)
    s1, tot = nve_energy_spread(oracle, pos, types, box, vel, 0.5, 10.0)
    s2, _ = nve_energy_spread(oracle, pos, types, box, vel, 0.25, 10.0)
    assert s1 < 3e-4 * abs(tot[0])
    assert 2.5 < s1 / s2 < 6.0


def test_per_atom_energies_sum_and_permute(oracle, hot):
    """Per-atom energies sum to the total, per term, and follow a relabelling
    of the atoms (the even split of each term does not depend on which atom
    of a pair is i)."""
    pos, types, box = hot
    for flags, k in ((FLAG_ALL, 0), (FLAG_REBO, 1), (FLAG_LJ, 2), (FLAG_TORSION, 3)):
        e, _, _, _, ea = oracle.compute(pos, types, box, flags, forces=False, per_atom=True)
        assert ea.sum() == pytest.approx(e[k], rel=1e-12, abs=1e-12)
    e, _, _, _, ea = oracle.compute(pos, types, box, per_atom=True)
    perm = np.random.default_rng(7).permutation(len(types))
    _, _, _, _, ea2 = oracle.compute(pos[:, perm], types[perm], box, per_atom=True)
    assert np.abs(ea2 - ea[perm]).max() < 1e-11 * np.abs(ea).max()
