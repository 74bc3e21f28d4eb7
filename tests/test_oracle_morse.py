"""AIREBO-M (Sec. 2.1.2: Morse in place of Lennard-Jones) in the oracle (no GPU)."""
import math

import numpy as np
import pytest

from paper_1810_07026_gb300 import inputs
from oracle.oracle import Oracle, FLAG_LJ, FLAG_ALL


@pytest.fixture(scope="module")
def morse_params():
    return inputs.make_params(0, morse=True)


@pytest.fixture(scope="module")
def morse_oracle(morse_params):
    return Oracle(inputs.params_text(morse_params))


def test_morse_between_molecules_closed_form(morse_oracle, morse_params):
    """Two H2 molecules 4 A apart: C = 1, S_r = 0, no cut-off switch, so the
    inter-molecular energy is the plain Morse sum eps (e^2 - 2e)."""
    p = morse_params
    a = np.array([[0, 0, 0], [0.74, 0, 0], [0, 4.0, 0.3], [0.74, 4.0, 0.3]]) + 20.0
    e, _, _, _ = morse_oracle.compute(np.ascontiguousarray(a.T), np.array([1, 1, 1, 1], dtype=np.int8),
                                      np.array([40.0, 40.0, 40.0]), FLAG_LJ)
    eps, alpha, re = p["morse.epsilon"][2], p["morse.alpha"][2], p["morse.re"][2]
    want = 0.0
    for i in (0, 1):
        for j in (2, 3):
            r = np.linalg.norm(a[i] - a[j])
            x = math.exp(-alpha * (r - re))
            want += eps * (x * x - 2 * x)
    assert e[2] == pytest.approx(want, rel=1e-12)


def test_morse_matches_lj_well(morse_params):
    """The default Morse term has the LJ well depth, minimum and curvature."""
    p = morse_params
    for k in range(3):
        sg, eps = p["lj.sigma"][k], p["lj.epsilon"][k]
        rm = 2 ** (1 / 6) * sg
        assert p["morse.re"][k] == pytest.approx(rm)
        assert p["morse.epsilon"][k] == pytest.approx(eps)
        assert 2 * eps * p["morse.alpha"][k] ** 2 == pytest.approx(72 * eps / rm ** 2)


def test_morse_forces_are_energy_gradient(morse_oracle):
    pos, types, box = inputs.amorphous(160, 1.0, 1.0, seed=11)
    _, f, _, _ = morse_oracle.compute(pos, types, box, FLAG_ALL)
    h = 1e-5
    worst = 0.0
    for a in range(0, 160, 23):
        for d in range(3):
            p = pos.copy(); p[d, a] += h
            ep = morse_oracle.energy(p, types, box)
            p[d, a] -= 2 * h
            em = morse_oracle.energy(p, types, box)
            worst = max(worst, abs(-(ep - em) / (2 * h) - f[d, a]))
    assert worst <= 2e-6 * np.abs(f).max()
