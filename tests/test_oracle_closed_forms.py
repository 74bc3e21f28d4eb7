"""Closed-form pins of the CPU oracle (no GPU).

Each case is a small molecule in a large box whose energy can be written out
by hand from the terms of Sec. 2.1 (E^REBO = f_R + b f_A, Alg. 1; b_ij =
1/2 (p_ij + p_ji) + pi^rc + pi^dh and p^{sigma pi}, Sec. 2.1.3; C_ij,
Sec. 2.1.2; torsion, Alg. 2) with every spline argument placed on a knot, so
the expected value uses only the knot data of the parameter set.  A dropped
term, a wrong sign, a swapped spline argument or a product in place of the
sum of p_ij and p_ji fails one of them.
"""
import math

import numpy as np
import pytest

from paper_1810_07026_gb300 import inputs
from oracle.oracle import Oracle, FLAG_REBO, FLAG_LJ, FLAG_TORSION

BOX = np.array([40.0, 40.0, 40.0])
CC, CH, HH = 0, 1, 2


def S(t):
    if t <= 0:
        return 1.0
    if t >= 1:
        return 0.0
    return 0.5 * (1.0 + math.cos(math.pi * t))


def w(p, pair, r):
    return S((r - p["Dmin"][pair]) / (p["Dmax"][pair] - p["Dmin"][pair]))


def fR(p, pair, r):
    return w(p, pair, r) * (1.0 + p["Q"][pair] / r) * p["A"][pair] * math.exp(-p["alpha"][pair] * r)


def fA(p, pair, r):
    s = sum(p[f"B{n}"][pair] * math.exp(-p[f"beta{n}"][pair] * r) for n in (1, 2, 3))
    return -w(p, pair, r) * s


def knot_P(p, tab, nc, nh):
    return p[f"P.{tab}"].reshape(5, 5, 4)[nc, nh, 0]


def knot_tri(p, name, a, b, nconj):
    return p[name].reshape(5, 5, 9, 8)[a, b, nconj - 1, 0]


def knot_g(p, name, idx):
    return p[f"{name}.data"].reshape(-1, 3)[idx, 0]


def run(oracle, atoms, types, flags=7):
    pos = np.ascontiguousarray(np.array(atoms, dtype=np.float64).T + 20.0)
    e, f, _, _ = oracle.compute(pos, np.array(types, dtype=np.int8), BOX, flags)
    return e, f


def test_h2_equilibrium(oracle, params):
    p, r = params, 0.74
    b = 0.5 * (1.0 + 1.0) + knot_tri(p, "piRC.HH", 0, 0, 1)
    e, _ = run(oracle, [[0, 0, 0], [r, 0, 0]], [1, 1])
    assert e[0] == pytest.approx(fR(p, HH, r) + b * fA(p, HH, r), rel=1e-13, abs=1e-13)
    assert e[2] == 0.0 and e[3] == 0.0


def test_h2_switched_bond_and_lj(params):
    """r inside the w switch: w enters f_R and f_A; C = 1 - w; with b* below
    b_min the LJ switch factor S_r S_b + 1 - S_r is 1 (S_r = 1 at r < sigma)."""
    p = {k: v.copy() for k, v in params.items()}
    d = p["piRC.HH"].reshape(5, 5, 9, 8)
    d[0, 0, 0, 0] = -0.8                        # b* = 1 - 0.8 = 0.2 < b_min(HH)
    o = Oracle(inputs.params_text(p))
    r = 1.45
    b = 1.0 - 0.8
    sg, eps = p["lj.sigma"][HH], p["lj.epsilon"][HH]
    vlj = 4 * eps * ((sg / r) ** 12 - (sg / r) ** 6)
    e, _ = run(o, [[0, 0, 0], [r, 0, 0]], [1, 1])
    assert e[1] == pytest.approx(fR(p, HH, r) + b * fA(p, HH, r), rel=1e-13)
    assert e[2] == pytest.approx((1.0 - w(p, HH, r)) * vlj, rel=1e-12)


def test_ch_radical(oracle, params):
    p, r = params, 1.1
    b = 1.0 + knot_tri(p, "piRC.CH", 0, 0, 1)
    e, _ = run(oracle, [[0, 0, 0], [r, 0, 0]], [0, 1])
    assert e[0] == pytest.approx(fR(p, CH, r) + b * fA(p, CH, r), rel=1e-13)


def test_ch2_bent_120(oracle, params):
    """H-C-H at 120 degrees: g_C = gamma_C (N = 1 < 3.2), P_CH(0, 1), F_CH(1, 0, 1)."""
    p, r = params, 1.09
    c, s = -0.5, math.sqrt(3) / 2
    pcs = (1.0 + knot_g(p, "gC2", 2) + knot_P(p, "CH", 0, 1)) ** -0.5
    b = 0.5 * (pcs + 1.0) + knot_tri(p, "piRC.CH", 1, 0, 1)
    e, _ = run(oracle, [[0, 0, 0], [r, 0, 0], [r * c, r * s, 0]], [0, 1, 1])
    assert e[0] == pytest.approx(2 * (fR(p, CH, r) + b * fA(p, CH, r)), rel=1e-12)
    assert e[2] == 0.0


def test_hhh_linear_lambda(oracle, params):
    """H-H-H: lambda_jik = 4 [(rho_kH - r_ik) - (rho_jH - r_ij)] for an H centre."""
    p = params
    r12, r23 = 0.9, 1.0
    gm1 = knot_g(p, "gH", 0)
    p21 = (1.0 + gm1 * math.exp(4 * (r12 - r23))) ** -0.5
    p23 = (1.0 + gm1 * math.exp(4 * (r23 - r12))) ** -0.5
    b12 = 0.5 * (1.0 + p21) + knot_tri(p, "piRC.HH", 0, 1, 1)
    b23 = 0.5 * (p23 + 1.0) + knot_tri(p, "piRC.HH", 1, 0, 1)
    expect = fR(p, HH, r12) + b12 * fA(p, HH, r12) + fR(p, HH, r23) + b23 * fA(p, HH, r23)
    e, _ = run(oracle, [[0, 0, 0], [r12, 0, 0], [r12 + r23, 0, 0]], [1, 1, 1])
    assert e[0] == pytest.approx(expect, rel=1e-12)


def test_c3_bent_conjugation(oracle, params):
    """C-C-C at 120 degrees: N^conj = 1 + A^2 + B^2 with A = 1, B = 0."""
    p, r = params, 1.4
    c, s = -0.5, math.sqrt(3) / 2
    p12 = (1.0 + knot_g(p, "gC2", 2) + knot_P(p, "CC", 1, 0)) ** -0.5
    b = 0.5 * (p12 + 1.0) + knot_tri(p, "piRC.CC", 1, 0, 2)
    e, _ = run(oracle, [[0, 0, 0], [r, 0, 0], [r * c, r * s, 0]], [0, 0, 0])
    assert e[0] == pytest.approx(2 * (fR(p, CC, r) + b * fA(p, CC, r)), rel=1e-12)
    assert e[3] == 0.0 and e[2] == 0.0


def hcch(dihedral_deg, rcc=1.4, rch=1.09):
    c1 = np.array([0.0, 0.0, 0.0])
    c2 = np.array([rcc, 0.0, 0.0])
    h1 = c1 + rch * np.array([-0.5, math.sqrt(3) / 2, 0.0])
    phi = math.radians(dihedral_deg)
    h2 = c2 + rch * np.array([0.5, math.sqrt(3) / 2 * math.cos(phi), math.sqrt(3) / 2 * math.sin(phi)])
    return [c1, c2, h1, h2], [0, 0, 1, 1]


def test_hcch_twisted_dihedral_and_torsion(oracle, params):
    """H-C-C-H twisted by 90 degrees: pi^dh = T_CC(1, 1, 1) (1 - cos^2 omega) with
    cos omega = 0, torsion V = eps_HCCH (256/405 (1/2)^5 - 1/10)."""
    p = params
    rcc, rch = 1.4, 1.09
    atoms, types = hcch(90.0, rcc, rch)
    pcc = (1.0 + knot_g(p, "gC2", 2) + knot_P(p, "CC", 0, 1)) ** -0.5
    bcc = pcc + knot_tri(p, "piRC.CC", 1, 1, 1) + knot_tri(p, "Tij.CC", 1, 1, 1)
    pch = (1.0 + knot_g(p, "gC2", 2) + knot_P(p, "CH", 1, 0)) ** -0.5
    bch = 0.5 * (pch + 1.0) + knot_tri(p, "piRC.CH", 1, 0, 2)
    erebo = fR(p, CC, rcc) + bcc * fA(p, CC, rcc) + 2 * (fR(p, CH, rch) + bch * fA(p, CH, rch))
    etors = p["tors.epsilon"][2] * (256.0 / 405.0 / 32.0 - 0.1)
    e, _ = run(oracle, atoms, types)
    assert knot_tri(p, "Tij.CC", 1, 1, 1) != 0.0
    assert e[1] == pytest.approx(erebo, rel=1e-12)
    assert e[3] == pytest.approx(etors, rel=1e-12)
    assert e[2] == 0.0


@pytest.mark.parametrize("dihedral,h5", [(180.0, 0.0), (0.0, 1.0)])
def test_torsion_trans_cis(oracle, params, dihedral, h5):
    """Trans (omega = pi) is the minimum -eps/10, cis gives eps (256/405 - 1/10)."""
    atoms, types = hcch(dihedral)
    e, _ = run(oracle, atoms, types, FLAG_TORSION)
    eps = params["tors.epsilon"][2]
    assert e[3] == pytest.approx(eps * (256.0 / 405.0 * h5 - 0.1), rel=1e-12, abs=1e-15)


def test_lj_plain_between_molecules(oracle, params):
    """Two H2 molecules 4 A apart: beyond three bonds (C = 1) and beyond
    2^(1/6) sigma (S_r = 0), so E^LJ is the plain LJ sum."""
    p = params
    a = [[0, 0, 0], [0.74, 0, 0], [0, 4.0, 0.3], [0.74, 4.0, 0.3]]
    e, _ = run(oracle, a, [1, 1, 1, 1], FLAG_LJ)
    sg, eps = p["lj.sigma"][HH], p["lj.epsilon"][HH]
    x = np.array(a)
    expect = 0.0
    for i in (0, 1):
        for j in (2, 3):
            r = np.linalg.norm(x[i] - x[j])
            expect += 4 * eps * ((sg / r) ** 12 - (sg / r) ** 6)
    assert e[2] == pytest.approx(expect, rel=1e-12)


def test_lj_cutoff_switch(oracle, params):
    """Beyond 2.7 sigma the LJ term is multiplied by 1 - 3t^2 + 2t^3."""
    p = params
    sg, eps = p["lj.sigma"][CC], p["lj.epsilon"][CC]
    r = 2.85 * sg
    t = (r - 2.7 * sg) / (0.3 * sg)
    e, _ = run(oracle, [[0, 0, 0], [r, 0, 0]], [0, 0], FLAG_LJ)
    assert e[2] == pytest.approx(4 * eps * ((sg / r) ** 12 - (sg / r) ** 6) * (1 - 3 * t * t + 2 * t ** 3), rel=1e-12)
    e, _ = run(oracle, [[0, 0, 0], [3.0 * sg + 1e-9, 0, 0]], [0, 0], FLAG_LJ)
    assert e[2] == 0.0


def test_cij_single_switched_bond(oracle, params):
    """H-C-C-H with the C-C bond in its switch: every 2- and 3-bond pair has
    C_ij = 1 - w_CC (all C-H weights are 1)."""
    p = params
    rcc = 1.85
    atoms, types = hcch(180.0, rcc=rcc)
    pos = np.ascontiguousarray(np.array(atoms).T + 20.0)
    oracle.rebo_neighbors(pos, np.array(types, dtype=np.int8), BOX)
    wcc = w(p, CC, rcc)
    assert 0.0 < wcc < 1.0
    for i, j in [(2, 3), (2, 1), (0, 3), (0, 1)]:
        c, path = oracle.cij(i, j, [0, 0, 0])
        assert c == pytest.approx(1.0 - wcc, rel=1e-14)
    c, path = oracle.cij(0, 2, [0, 0, 0])       # direct C-H bond with w = 1
    assert c == 0.0 and path[0] == 1
