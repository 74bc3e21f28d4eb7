"""Seeded synthetic inputs shared by the CUDA path, the tests and the bench.

This module holds no arithmetic of the AIREBO method itself.  It only draws
seeded random numbers and lays out:

* the parameter set (scalars of the REBO pair terms, the LJ term, the torsion
  term and the switches, plus the knot data of every spline), written as the
  plain-text parameter file that ``airebo_create`` and the CPU oracle each
  parse on their own;
* the atomic systems of the workloads: a noisy diamond-cubic carbon crystal,
  crystalline polyethylene (PE) built from zig-zag CH2 chains, and amorphous
  C:H boxes filled by random sequential insertion;
* Maxwell-Boltzmann velocities.

The paper (Sec. 2.1) names the terms of AIREBO but prints none of its
parameter values or spline tables; the tables here are seeded smooth stand-ins
with the symmetries the method needs (F(a,b,c) = F(b,a,c) for the
same-species pi^rc and T tables, P(0,0) = 0).  The scalar defaults are the
commonly quoted values of the published potential; nothing here claims they
are exact.

Units are LAMMPS "metal": Angstrom, eV, fs, amu.  Arrays of positions and
velocities are structure-of-arrays, shape (3, N), float64.  Types are int8,
0 = carbon, 1 = hydrogen.
"""
from __future__ import annotations

import math
import numpy as np

MASS = (12.011, 1.008)          # amu, carbon and hydrogen
KB_EV = 8.617333262e-5          # Boltzmann constant, eV/K
MVV2E = 103.642697              # 1 amu*A^2/fs^2 in eV

PAIR_NAMES = ("CC", "CH", "HH")

# knot abscissae of the angular functions, in cos(theta)
GC_KNOTS = (-1.0, -2.0 / 3.0, -0.5, -1.0 / 3.0, 0.0, 1.0)
GH_KNOTS = (-1.0, -5.0 / 6.0, -0.5, 1.0)
# integer knot grids of the coordination splines
P_GRID = (5, 5)            # N^C, N^H in 0..4
TRI_GRID = (5, 5, 9)       # N_ij, N_ji in 0..4, N^conj in 1..9
TRI_ZMIN = 1.0


def _angular_data(rng, knots, a, b, jitter=0.03):
    """(value, first, second derivative) at each knot of a positive,
    increasing seeded function close to a*exp(b*(c+1))."""
    out = []
    for c in knots:
        e = a * math.exp(b * (c + 1.0))
        v = e * (1.0 + jitter * rng.uniform(-1, 1))
        d1 = a * b * math.exp(b * (c + 1.0)) * (1.0 + 0.05 * rng.uniform(-1, 1))
        d2 = a * b * b * math.exp(b * (c + 1.0)) * (1.0 + 0.05 * rng.uniform(-1, 1))
        out += [v, d1, d2]
    return np.array(out, dtype=np.float64)


def _bicubic_data(rng, scale, dscale, zero_origin=True):
    """Knot data f, f_x, f_y, f_xy on the 5x5 grid, index (x, y, component)."""
    d = np.zeros(P_GRID + (4,))
    d[..., 0] = rng.uniform(-scale, scale, P_GRID)
    d[..., 1] = rng.uniform(-dscale, dscale, P_GRID)
    d[..., 2] = rng.uniform(-dscale, dscale, P_GRID)
    d[..., 3] = rng.uniform(-dscale, dscale, P_GRID) * 0.5
    if zero_origin:
        d[0, 0, 0] = 0.0
    return d


# component order of tricubic knot data
TRI_COMPONENTS = ("f", "fx", "fy", "fz", "fxy", "fxz", "fyz", "fxyz")


def _symmetrize_xy(d):
    """Make knot data describe a function with F(a,b,c) = F(b,a,c).

    Components that are even under the swap of x and y are averaged with
    their transpose; f_x and f_y (and f_xz, f_yz) are exchanged by it."""
    t = np.swapaxes(d, 0, 1).copy()
    s = np.empty_like(d)
    for c in (0, 3, 4, 7):                   # f, fz, fxy, fxyz
        s[..., c] = 0.5 * (d[..., c] + t[..., c])
    s[..., 1] = 0.5 * (d[..., 1] + t[..., 2])  # fx(a,b) <-> fy(b,a)
    s[..., 2] = np.swapaxes(s[..., 1], 0, 1)
    s[..., 5] = 0.5 * (d[..., 5] + t[..., 6])  # fxz <-> fyz
    s[..., 6] = np.swapaxes(s[..., 5], 0, 1)
    return s


def _tricubic_data(rng, scale, dscale, symmetric):
    d = np.zeros(TRI_GRID + (8,))
    d[..., 0] = rng.uniform(-scale, scale, TRI_GRID)
    for c in range(1, 8):
        d[..., c] = rng.uniform(-dscale, dscale, TRI_GRID) * (0.5 if c >= 4 else 1.0)
    if symmetric:
        d = _symmetrize_xy(d)
    return d


def _dihedral_data(rng, scale, dscale):
    """Seeded T_CC knot data, nonzero only at knots with N_ij and N_ji in {1, 2}.

    So T vanishes, with its gradient, wherever either carbon has three or more
    other neighbours: saturated crystals skip the dihedral sum, the
    under-coordinated atoms of amorphous inputs exercise it."""
    d = np.zeros(TRI_GRID + (8,))
    mask = np.zeros(TRI_GRID, dtype=bool)
    mask[1:3, 1:3, :] = True
    d[..., 0] = np.where(mask, rng.uniform(-scale, 0.0, TRI_GRID), 0.0)
    for c in range(1, 8):
        d[..., c] = np.where(mask, rng.uniform(-dscale, dscale, TRI_GRID), 0.0)
    return _symmetrize_xy(d)


def make_params(seed: int = 0, morse: bool = False) -> dict:
    """The full parameter set: scalars (per type pair CC, CH, HH) and seeded tables.

    morse=True selects the AIREBO-M form of the inter-molecular term: a Morse
    potential whose well depth, minimum and curvature equal those of the LJ
    term (r_e = 2^(1/6) sigma, alpha = 6 / r_e)."""
    rng = np.random.default_rng(seed)
    p = {}
    p["Dmin"] = [1.7, 1.3, 1.1]
    p["Dmax"] = [2.0, 1.8, 1.7]
    p["Q"] = [0.3134602960833, 0.340775728, 0.370471487045]
    p["alpha"] = [4.7465390606595, 4.10254983, 3.536298648]
    p["A"] = [10953.544162170, 149.94098723, 32.817355747]
    p["B1"] = [12388.79197798, 32.3551866587, 29.632593]
    p["B2"] = [17.56740646509, 0.0, 0.0]
    p["B3"] = [30.71493208065, 0.0, 0.0]
    p["beta1"] = [4.7204523127, 1.43445805925, 1.71589217]
    p["beta2"] = [1.4332132499, 0.0, 0.0]
    p["beta3"] = [1.3826912506, 0.0, 0.0]
    p["rho"] = [0.0, 1.09, 0.7415887]
    p["lambda_coef"] = [4.0]
    p["gC_Nswitch"] = [3.2, 3.7]
    p["Fconj_x"] = [2.0, 3.0]
    p["gC1.knots"] = list(GC_KNOTS)
    p["gC1.data"] = _angular_data(rng, GC_KNOTS, 0.02, 3.0)
    p["gC2.knots"] = list(GC_KNOTS)
    p["gC2.data"] = _angular_data(rng, GC_KNOTS, 0.03, 2.8)
    p["gH.knots"] = list(GH_KNOTS)
    p["gH.data"] = _angular_data(rng, GH_KNOTS, 0.8, 1.5)
    p["P.CC"] = _bicubic_data(rng, 0.05, 0.02)
    p["P.CH"] = _bicubic_data(rng, 0.05, 0.02)
    p["P.HC"] = _bicubic_data(rng, 0.05, 0.02)
    p["piRC.CC"] = _tricubic_data(rng, 0.1, 0.03, symmetric=True)
    p["piRC.CH"] = _tricubic_data(rng, 0.1, 0.03, symmetric=False)
    p["piRC.HH"] = _tricubic_data(rng, 0.1, 0.03, symmetric=True)
    p["Tij.CC"] = _dihedral_data(rng, 0.04, 0.02)
    p["dihedral_guard"] = [0.995, 0.005]
    p["lj.sigma"] = [3.40, 3.025, 2.65]
    p["lj.epsilon"] = [0.00284, math.sqrt(0.00284 * 0.00150), 0.00150]
    p["lj.cut"] = [3.0]
    p["lj.switch_start"] = [2.7]
    p["lj.Sr_range"] = [1.0, 2.0 ** (1.0 / 6.0)]
    p["bstar.bmin"] = [0.77, 0.75, 0.32]
    p["bstar.bmax"] = [0.81, 0.90, 0.42]
    p["bstar.rstar"] = list(p["Dmin"])
    p["tors.epsilon"] = [0.3079, 0.1787, 0.1250]
    p["inter.kind"] = [1.0 if morse else 0.0]
    re = [2.0 ** (1.0 / 6.0) * s for s in p["lj.sigma"]]
    p["morse.epsilon"] = list(p["lj.epsilon"])
    p["morse.re"] = re
    p["morse.alpha"] = [6.0 / x for x in re]
    return {k: np.asarray(v, dtype=np.float64).ravel() for k, v in p.items()}


def params_text(p: dict) -> str:
    """Serialise a parameter set: one line ``name count v1 v2 ...`` per entry."""
    lines = ["#AIREBO-PARAMS 1"]
    for k, v in p.items():
        vals = " ".join(repr(float(x)) for x in np.asarray(v).ravel())
        lines.append(f"{k} {np.asarray(v).size} {vals}")
    return "\n".join(lines) + "\n"


def write_params(path: str, p: dict | None = None, seed: int = 0) -> str:
    p = make_params(seed) if p is None else p
    with open(path, "w") as f:
        f.write(params_text(p))
    return path


# --------------------------------------------------------------------------
# systems
# --------------------------------------------------------------------------

def diamond(ncell: int = 3, a: float = 3.567, noise: float = 0.05, seed: int = 1):
    """Diamond-cubic carbon, ncell^3 conventional cells (8 atoms each)."""
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                      [.25, .25, .25], [.25, .75, .75], [.75, .25, .75], [.75, .75, .25]])
    cells = np.array([[i, j, k] for i in range(ncell) for j in range(ncell) for k in range(ncell)])
    frac = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    pos = frac * a
    rng = np.random.default_rng(seed)
    pos = pos + rng.normal(0.0, noise, pos.shape)
    box = np.array([ncell * a] * 3)
    types = np.zeros(len(pos), dtype=np.int8)
    return np.ascontiguousarray(pos.T), types, box


def polyethylene(nx: int, ny: int, nz: int, noise: float = 0.03, seed: int = 1,
                 a: float = 7.40, b: float = 4.93, c: float = 2.54,
                 r_cc: float = 1.54, r_ch: float = 1.09, setting_deg: float = 42.0):
    """Orthorhombic crystalline PE: two CH2 zig-zag chains per cell along z.

    Each cell repeat holds two carbons per chain; the zig-zag plane of the
    chain at the cell corner is rotated by +setting_deg about z, the one at the
    face centre by -setting_deg.  Hydrogens sit in the plane normal to the
    zig-zag plane with an H-C-H angle of 109.47 degrees."""
    half = 0.5 * c
    lateral = math.sqrt(r_cc * r_cc - half * half)     # zig-zag amplitude
    th = math.radians(109.4712206 / 2.0)
    # the 12 atoms of one cell, relative to the cell corner
    motif, mtypes = [], []
    chains = [((0.0, 0.0), +setting_deg), ((0.5 * a, 0.5 * b), -setting_deg)]
    for (cx, cy), phi in chains:
        u = np.array([math.cos(math.radians(phi)), math.sin(math.radians(phi)), 0.0])
        v = np.array([-u[1], u[0], 0.0])
        for s, zoff in ((+1, 0.0), (-1, half)):
            C = np.array([cx, cy, zoff]) + s * 0.5 * lateral * u
            motif.append(C); mtypes.append(0)
            out = s * u
            for sv in (+1, -1):
                motif.append(C + r_ch * (math.cos(th) * out + sv * math.sin(th) * v))
                mtypes.append(1)
    motif = np.array(motif)
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    corners = np.stack([ix.ravel() * a, iy.ravel() * b, iz.ravel() * c], axis=1)
    atoms = (corners[:, None, :] + motif[None, :, :]).reshape(-1, 3)
    types = np.tile(np.array(mtypes), len(corners))
    pos = atoms
    box = np.array([nx * a, ny * b, nz * c])
    pos = np.mod(pos, box)
    rng = np.random.default_rng(seed)
    pos = pos + rng.normal(0.0, noise, pos.shape)
    return np.ascontiguousarray(pos.T), np.array(types, dtype=np.int8), box


def amorphous(n: int, h_per_c: float, density_gcc: float, seed: int = 1,
              min_sep: float = 1.0, max_tries: int = 2000):
    """Amorphous C:H box by seeded random sequential insertion (periodic)."""
    rng = np.random.default_rng(seed)
    nc = int(round(n / (1.0 + h_per_c)))
    types = np.zeros(n, dtype=np.int8)
    types[nc:] = 1
    rng.shuffle(types)
    mass = np.where(types == 0, MASS[0], MASS[1]).sum()
    vol = mass / 0.602214076 / density_gcc          # A^3 (1 g/cm^3 = 0.6022 amu/A^3)
    L = vol ** (1.0 / 3.0)
    box = np.array([L, L, L])
    pos = np.zeros((n, 3))
    placed = 0
    ms2 = min_sep * min_sep
    for t in range(n):
        for _ in range(max_tries):
            x = rng.uniform(0.0, L, 3)
            if placed == 0:
                break
            d = pos[:placed] - x
            d -= L * np.round(d / L)
            if np.min(np.einsum("ij,ij->i", d, d)) >= ms2:
                break
        else:
            raise RuntimeError("random insertion failed; density too high for min_sep")
        pos[placed] = x
        placed += 1
    return np.ascontiguousarray(pos.T), types, box


def amorphous_kd(n: int, h_per_c: float, density_gcc: float, seed: int = 1, min_sep: float = 1.0):
    """Amorphous C:H box by seeded random insertion with a minimum separation,
    accepting candidates in batches (a periodic KD-tree rejects those too close
    to accepted atoms or to earlier candidates of the same batch)."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    nc = int(round(n / (1.0 + h_per_c)))
    types = np.zeros(n, dtype=np.int8)
    types[nc:] = 1
    rng.shuffle(types)
    mass = np.where(types == 0, MASS[0], MASS[1]).sum()
    L = (mass / 0.602214076 / density_gcc) ** (1.0 / 3.0)
    acc = np.zeros((0, 3))
    for _ in range(200):
        need = n - len(acc)
        if need == 0:
            break
        cand = rng.uniform(0.0, L, (max(2 * need, 64), 3))
        if len(acc):
            dist, _ = cKDTree(acc, boxsize=L).query(cand, k=1, distance_upper_bound=min_sep)
            cand = cand[~np.isfinite(dist)]
        keep = np.ones(len(cand), dtype=bool)
        if len(cand) > 1:
            for i, j in sorted(cKDTree(cand, boxsize=L).query_pairs(min_sep)):
                if keep[i] and keep[j]:
                    keep[j] = False
        acc = np.vstack([acc, cand[keep][:need]])
    if len(acc) < n:
        raise RuntimeError("random insertion failed; density too high for min_sep")
    return np.ascontiguousarray(acc.T), types, np.array([L, L, L])


def ensemble(nsys: int = 256, nmin: int = 200, nmax: int = 8000, density_gcc: float = 0.9,
             hc: tuple = (0.5, 2.0), seed: int = 7):
    """Independent amorphous C:H boxes of uneven size, concatenated: positions
    (3, N), types (N,), offsets (nsys + 1,), boxes (nsys, 3)."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(nmin, nmax + 1, nsys)
    ratios = rng.uniform(hc[0], hc[1], nsys)
    pos, typ, boxes = [], [], []
    for s in range(nsys):
        p, t, b = amorphous_kd(int(sizes[s]), float(ratios[s]), density_gcc, seed=seed * 100003 + s)
        pos.append(p); typ.append(t); boxes.append(b)
    offsets = np.concatenate([[0], np.cumsum([len(t) for t in typ])]).astype(np.int64)
    return np.ascontiguousarray(np.hstack(pos)), np.concatenate(typ), offsets, np.array(boxes)


def velocities(types, temperature: float, seed: int = 2):
    """Maxwell-Boltzmann velocities in A/fs with zero total momentum."""
    rng = np.random.default_rng(seed)
    m = np.where(np.asarray(types) == 0, MASS[0], MASS[1])
    sd = np.sqrt(KB_EV * temperature / (m * MVV2E))
    v = rng.normal(0.0, 1.0, (3, len(m))) * sd
    p = (v * m).sum(axis=1) / m.sum()
    v -= p[:, None]
    return np.ascontiguousarray(v)


def masses(types):
    return np.where(np.asarray(types) == 0, MASS[0], MASS[1]).astype(np.float64)


WORKLOADS = {
    "diamond216": dict(kind="diamond", ncell=3, noise=0.05, seed=1),
    "pe32k": dict(kind="pe", cells=(17, 20, 8), noise=0.03, seed=1),
    "pe1m": dict(kind="pe", cells=(34, 40, 64), noise=0.05, seed=1),
    "pe261k": dict(kind="pe", cells=(34, 40, 16), noise=0.05, seed=1),
}


def workload(name: str):
    w = WORKLOADS[name]
    if w["kind"] == "diamond":
        return diamond(w["ncell"], noise=w["noise"], seed=w["seed"])
    nx, ny, nz = w["cells"]
    return polyethylene(nx, ny, nz, noise=w["noise"], seed=w["seed"])
