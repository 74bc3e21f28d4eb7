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


# ---------------------------------------------------------------------------
# pins of the switches that only act in their transitions: S_r and S_b of the
# LJ term with the fixed length of b* (Alg. 3, Sec. 2.1.3), the N-blend of the
# carbon angular function and the F(x_ik) switch of N^conj (Sec. 2.1.3), and
# the angle guard of the dihedral sums (torsion, Alg. 2, and pi^dh)
# ---------------------------------------------------------------------------

def _copy(params):
    return {k: v.copy() for k, v in params.items()}


def _constant_angular(p, name, value):
    """Knot data of an angular function that is the constant `value`
    (zero slope and curvature at every knot)."""
    d = p[f"{name}.data"].reshape(-1, 3)
    d[:, 0] = value
    d[:, 1:] = 0.0


def _flat_bond_order(p, g=0.1):
    """Angle-independent angular functions, P = 0, pi^rc = 0 and T = 0: the
    bond order then follows from the coordinations alone."""
    _constant_angular(p, "gC1", g)
    _constant_angular(p, "gC2", g)
    _constant_angular(p, "gH", g)
    for t in ("P.CC", "P.CH", "P.HC", "piRC.CC", "piRC.CH", "piRC.HH", "Tij.CC"):
        p[t][:] = 0.0


def test_lj_bstar_transition_and_rstar(params):
    """An H-H LJ pair (i, j) with sigma < r_ij < 2^(1/6) sigma, i bonded to a
    third H k: S_r and S_b are both fractional, C_ij = 1.  b* is the bond
    order at the fixed length r* = Dmin_HH along r_ij, so lambda_jik =
    4 (r* - r_ik); pi^rc_HH(1, 0, 1) is set so that this b* lands in the middle
    of [b_min, b_max].  With |r_ij| in place of r* (the b* bug of Sec. 3.3),
    lambda is 4 (r_ij - r_ik), b* is far below b_min and S_b = 1."""
    p = _copy(params)
    sg, eps = p["lj.sigma"][HH], p["lj.epsilon"][HH]
    rstar = p["bstar.rstar"][HH]
    assert rstar == p["Dmin"][HH]
    r, rik = 2.8, 0.74
    assert sg < r < 2 ** (1 / 6) * sg
    lam = p["lambda_coef"][0] * ((p["rho"][HH] - rik) - (p["rho"][HH] - rstar))
    g = knot_g(p, "gH", 2)                           # cos(theta_jik) = -1/2
    p_ij = (1.0 + g * math.exp(lam)) ** -0.5
    b_target = 0.5 * (p["bstar.bmin"][HH] + p["bstar.bmax"][HH])
    F = b_target - 0.5 * (p_ij + 1.0)
    d = p["piRC.HH"].reshape(5, 5, 9, 8)
    d[1, 0, 0, 0] = d[0, 1, 0, 0] = F                # keeps F(a, b, c) = F(b, a, c)
    o = Oracle(inputs.params_text(p))
    xk = [rik * -0.5, rik * math.sqrt(3) / 2, 0.0]
    atoms = [[0, 0, 0], [r, 0, 0], xk]
    rkj = math.dist([r, 0, 0], xk)
    assert rkj > 2 ** (1 / 6) * sg                   # the k-j pair: S_r = 0, C = 1

    def vlj(x):
        return 4 * eps * ((sg / x) ** 12 - (sg / x) ** 6)

    Sr = S((r - sg) / ((2 ** (1 / 6) - 1) * sg))
    Sb = S((b_target - p["bstar.bmin"][HH]) / (p["bstar.bmax"][HH] - p["bstar.bmin"][HH]))
    assert 0.1 < Sr < 0.9 and Sb == pytest.approx(0.5, abs=1e-12)
    e, _ = run(o, atoms, [1, 1, 1], FLAG_LJ)
    assert e[2] == pytest.approx((Sr * Sb + 1.0 - Sr) * vlj(r) + vlj(rkj), rel=1e-11)


def test_gC_coordination_blend(params):
    """A carbon with five carbon neighbours (trigonal bipyramid, one axial bond
    in its w switch, w = 1/2): for each full bond N_ij = 3.5 lies inside the
    switch Q(N) = S((N - 3.2)/0.5), so g_C = G_C + Q (gamma_C - G_C) blends the
    two angular functions (made constant here, G_C = 0.05, gamma_C = 0.2); for
    the switched bond N_ij = 4 and g_C = G_C.  P, pi^rc, pi^dh are zero, so b =
    (1/2)[(1 + N g_C(N))^(-1/2) + 1] for every bond."""
    p = _copy(params)
    _flat_bond_order(p)
    G, gam = 0.05, 0.2
    _constant_angular(p, "gC1", G)
    _constant_angular(p, "gC2", gam)
    o = Oracle(inputs.params_text(p))
    r0, r5 = 1.54, 1.85
    w5 = w(p, CC, r5)
    assert w5 == pytest.approx(0.5, abs=1e-12)
    atoms = [[0, 0, 0], [r0, 0, 0], [-0.5 * r0, math.sqrt(3) / 2 * r0, 0], [-0.5 * r0, -math.sqrt(3) / 2 * r0, 0],
             [0, 0, r0], [0, 0, -r5]]
    x = np.array(atoms)
    for a in range(1, 6):
        for b in range(a + 1, 6):
            assert np.linalg.norm(x[a] - x[b]) > p["Dmax"][CC]

    def gC(N):
        return G + S((N - 3.2) / 0.5) * (gam - G)

    expect = 0.0
    for rb, N in [(r0, 3.0 + w5)] * 4 + [(r5, 4.0)]:
        b = 0.5 * ((1.0 + N * gC(N)) ** -0.5 + 1.0)
        expect += fR(p, CC, rb) + b * fA(p, CC, rb)
    assert 0.0 < S((3.0 + w5 - 3.2) / 0.5) < 1.0
    e, _ = run(o, atoms, [0] * 6, FLAG_REBO)
    assert e[1] == pytest.approx(expect, rel=1e-12)


def test_conjugation_F_transition(params):
    """j - i - k carbons with k saturated by two H at full weight and one H in
    its C-H switch (w = 1/2): x_ik = N_k - w_ik = 2.5 is inside the switch
    F(x) = S(x - 2), F = 1/2.  pi^rc_CC is made linear in its third argument,
    pi^rc_CC = s N^conj, so it reads N^conj = 1 + (w_ik F(x_ik))^2 = 1.25 on
    bond i-j and 1 + (w_ij F(x_ij))^2 = 2 (x_ij = 0) on bond i-k.  The other
    bond-order parts are flat (constant g, P = 0, pi^rc_CH = 0, T = 0)."""
    p = _copy(params)
    g = 0.1
    _flat_bond_order(p, g)
    s = 0.01
    d = p["piRC.CC"].reshape(5, 5, 9, 8)
    d[..., 0] = s * (np.arange(9) + 1.0)[None, None, :]
    d[..., 3] = s
    o = Oracle(inputs.params_text(p))
    rcc, rch, rsw = 1.54, 1.09, 1.55
    wsw = w(p, CH, rsw)
    assert wsw == pytest.approx(0.5, abs=1e-12)
    k = np.array([rcc, 0.0, 0.0])
    dirs = [np.array([1 / 3, 2 * math.sqrt(2) / 3 * math.cos(f), 2 * math.sqrt(2) / 3 * math.sin(f)])
            for f in (0.0, 2 * math.pi / 3, 4 * math.pi / 3)]
    atoms = [[0, 0, 0], [-0.5 * rcc, math.sqrt(3) / 2 * rcc, 0], k,
             k + rch * dirs[0], k + rch * dirs[1], k + rsw * dirs[2]]
    types = [0, 0, 0, 1, 1, 1]
    x = np.array(atoms)
    bonded = {(0, 1), (0, 2), (2, 3), (2, 4), (2, 5)}
    for a in range(6):
        for b in range(a + 1, 6):
            if (a, b) not in bonded:
                pair = types[a] + types[b]
                assert np.linalg.norm(x[a] - x[b]) > p["Dmax"][pair]
    Nk = 1.0 + 1.0 + 1.0 + wsw
    F = S(Nk - 1.0 - 2.0)
    assert F == pytest.approx(0.5, abs=1e-12)
    b_ij = 0.5 * ((1.0 + g) ** -0.5 + 1.0) + s * (1.0 + F ** 2)
    b_ik = 0.5 * ((1.0 + g) ** -0.5 + (1.0 + (Nk - 1.0) * g) ** -0.5) + s * 2.0
    expect = fR(p, CC, rcc) + b_ij * fA(p, CC, rcc) + fR(p, CC, rcc) + b_ik * fA(p, CC, rcc)
    for rh, wh in ((rch, 1.0), (rch, 1.0), (rsw, wsw)):
        b = 0.5 * ((1.0 + (Nk - wh) * g) ** -0.5 + 1.0)
        expect += fR(p, CH, rh) + b * fA(p, CH, rh)
    e, _ = run(o, atoms, types, FLAG_REBO)
    assert e[1] == pytest.approx(expect, rel=1e-12)


def test_angle_guard_in_torsion_and_dihedral(params):
    """H-C-C-H twisted by 90 degrees with one H nearly collinear with the C-C
    bond, cos(theta) = -0.997: the guard s = S((|cos| - 0.995)/0.005) = S(0.4)
    scales the torsion term and the pi^dh sum; the other H sits at 120
    degrees, s = 1.  With constant angular functions the bond orders follow
    from knot data alone."""
    p = _copy(params)
    g = 0.1
    _constant_angular(p, "gC1", g)
    _constant_angular(p, "gC2", g)
    o = Oracle(inputs.params_text(p))
    rcc, rch, ca = 1.4, 1.09, 0.997
    sa = math.sqrt(1.0 - ca * ca)
    atoms = [[0, 0, 0], [rcc, 0, 0], [-rch * ca, rch * sa, 0], [rcc + 0.5 * rch, 0, rch * math.sqrt(3) / 2]]
    types = [0, 0, 1, 1]
    sg = S((ca - p["dihedral_guard"][0]) / p["dihedral_guard"][1])
    assert 0.1 < sg < 0.9
    e, _ = run(o, atoms, types)
    etors = sg * p["tors.epsilon"][2] * (256.0 / 405.0 / 32.0 - 0.1)
    assert e[3] == pytest.approx(etors, rel=1e-11)
    pcc = (1.0 + g + knot_P(p, "CC", 0, 1)) ** -0.5
    bcc = pcc + knot_tri(p, "piRC.CC", 1, 1, 1) + knot_tri(p, "Tij.CC", 1, 1, 1) * sg
    pch = (1.0 + g + knot_P(p, "CH", 1, 0)) ** -0.5
    bch = 0.5 * (pch + 1.0) + knot_tri(p, "piRC.CH", 1, 0, 2)
    erebo = fR(p, CC, rcc) + bcc * fA(p, CC, rcc) + 2 * (fR(p, CH, rch) + bch * fA(p, CH, rch))
    assert knot_tri(p, "Tij.CC", 1, 1, 1) != 0.0
    assert e[1] == pytest.approx(erebo, rel=1e-11)


def test_per_atom_energy_split(oracle, params):
    """Per-atom energies split each term evenly between its two atoms: for two
    H2 molecules 4 A apart, each H holds half its molecule's bond energy
    (Alg. 1) and half of every LJ pair it is in (C = 1, S_r = 0 at 4 A)."""
    p = params
    a = [[0, 0, 0], [0.74, 0, 0], [0, 4.0, 0.3], [0.74, 4.0, 0.3]]
    pos = np.ascontiguousarray(np.array(a, dtype=np.float64).T + 20.0)
    e, _, _, _, ea = oracle.compute(pos, np.ones(4, dtype=np.int8), BOX, per_atom=True)
    sg, eps = p["lj.sigma"][HH], p["lj.epsilon"][HH]
    x = np.array(a)
    ebond = fR(p, HH, 0.74) + (1.0 + knot_tri(p, "piRC.HH", 0, 0, 1)) * fA(p, HH, 0.74)
    for i in range(4):
        others = (2, 3) if i < 2 else (0, 1)
        lj = sum(4 * eps * ((sg / r) ** 12 - (sg / r) ** 6) for r in (np.linalg.norm(x[i] - x[j]) for j in others))
        assert ea[i] == pytest.approx(0.5 * ebond + 0.5 * lj, rel=1e-12)
    assert ea.sum() == pytest.approx(e[0], rel=1e-13)
