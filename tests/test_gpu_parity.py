"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (FP64 path, and the DF64 path whose LJ pair arithmetic runs in
double-float): |dE| <= 1e-10 |E|, max|dF| <= 1e-8 max|F|,
max|dW| <= 1e-8 max|W| -- the bar for a potential whose every term is
evaluated in double precision (differences come only from the order of
floating-point sums and from FP64 atomics).  Mixed path: FP32
geometry/splines/bond order against FP64 gives about 1e-6 relative per term;
the test allows |dE| <= 1e-6 (|E_REBO| + |E_LJ| + |E_tors|) and
max|dF| <= 2e-5 max|F|.
"""
import numpy as np
import pytest

from paper_1810_07026_gb300 import inputs
from oracle.oracle import FLAG_REBO, FLAG_LJ, FLAG_TORSION, FLAG_ALL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def A():
    from paper_1810_07026_gb300 import build, airebo
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return airebo


CASES = {
    "diamond216": lambda: inputs.diamond(),
    "pe1152": lambda: inputs.polyethylene(3, 4, 8, noise=0.05),
    "hot160": lambda: inputs.amorphous(160, 1.0, 1.0, seed=11),
    "hot300": lambda: inputs.amorphous(300, 0.5, 0.9, seed=5),
    "hot1000": lambda: inputs.amorphous(1000, 1.5, 0.9, seed=7),
}
FLAGS = {"all": FLAG_ALL, "rebo": FLAG_REBO, "lj": FLAG_LJ, "torsion": FLAG_TORSION}


def gpu_eval(A, params, pos, types, box, flags=FLAG_ALL, precision=0, virial=True, **kw):
    ev = A.Airebo(params, precision=precision, rebo=bool(flags & 1), lj=bool(flags & 2),
                  torsion=bool(flags & 4), **kw)
    p = torch.tensor(pos, device="cuda")
    ev.neighbor(p, torch.tensor(types, device="cuda"), box)
    f, e4, w6 = ev.compute(p, virial=virial)
    torch.cuda.synchronize()
    out = (e4.cpu().numpy(), f.cpu().numpy(), w6.cpu().numpy() if virial else None)
    return out, ev


def assert_close(got, want, etol, ftol, wtol=None, escale="total"):
    """escale "total": energies within etol |E_total|; "terms": within etol
    (|E_REBO| + |E_LJ| + |E_tors|), the scale of rounding errors when the
    terms cancel (hot boxes whose repulsive LJ energy offsets the REBO one)."""
    eg, fg, wg = got
    ew, fw, ww = want
    es = abs(ew[0]) if escale == "total" else abs(ew[1]) + abs(ew[2]) + abs(ew[3])
    assert abs(eg[0] - ew[0]) <= etol * max(es, 1e-12), (eg, ew)
    for k in (1, 2, 3):
        assert abs(eg[k] - ew[k]) <= etol * max(es, 1e-12) + 1e-12, (k, eg, ew)
    fs = max(np.abs(fw).max(), 1e-12)
    assert np.abs(fg - fw).max() <= ftol * fs, np.abs(fg - fw).max() / fs
    if wtol is not None and wg is not None:
        assert np.abs(wg - ww).max() <= wtol * max(np.abs(ww).max(), 1e-12)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("term", list(FLAGS))
def test_fp64_parity(A, oracle, param_text, case, term):
    pos, types, box = CASES[case]()
    flags = FLAGS[term]
    e, f, w, _ = oracle.compute(pos, types, box, flags)
    got, _ = gpu_eval(A, param_text, pos, types, box, flags)
    assert_close(got, (e, f, w), 1e-10, 1e-8, 1e-8)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("term", list(FLAGS))
def test_df64_parity(A, oracle, param_text, case, term):
    """DF64 (LJ pair and torsion arithmetic in double-float) against the
    oracle, term by term, at the FP64 tolerances."""
    pos, types, box = CASES[case]()
    flags = FLAGS[term]
    e, f, w, _ = oracle.compute(pos, types, box, flags)
    got, _ = gpu_eval(A, param_text, pos, types, box, flags, precision=A.DF64)
    assert_close(got, (e, f, w), 1e-10, 1e-8, 1e-8)


def test_df64_against_fp64_pe32k(A, param_text):
    """DF64 against FP64 on the 32,640-atom PE: the LJ pair and torsion
    arithmetic in double-float and the fixed-point LJ force sums stay within
    1e-11 of FP64."""
    pos, types, box = inputs.workload("pe32k")
    (e64, f64, w64), _ = gpu_eval(A, param_text, pos, types, box)
    (edf, fdf, wdf), _ = gpu_eval(A, param_text, pos, types, box, precision=A.DF64)
    assert abs(edf[0] - e64[0]) <= 1e-11 * abs(e64[0])
    assert np.abs(fdf - f64).max() <= 1e-11 * np.abs(f64).max()
    assert np.abs(wdf - w64).max() <= 1e-11 * np.abs(w64).max()


def test_df64_coordinate_range(A, param_text):
    pos, types, box = CASES["pe1152"]()
    assert (2100.0 / box).max() < 120          # still a valid position for the list build
    ev = A.Airebo(param_text, precision=A.DF64)
    p = torch.tensor(pos + 2100.0, device="cuda")
    ev.neighbor(p, torch.tensor(types, device="cuda"), box)
    with pytest.raises(A.AireboError):
        ev.compute(p)


@pytest.mark.parametrize("case", list(CASES))
def test_mixed_parity(A, oracle, param_text, case):
    """Mixed path: every energy within 1e-6 of the terms' scale |E_REBO| +
    |E_LJ| + |E_tors| (the total cancels in hot boxes: 216 eV of LJ against
    -161 eV of REBO in hot160), max|dF| <= 2e-5 max|F|; FP32 arithmetic in the
    geometry, splines and bond order gives about 1e-6 relative."""
    pos, types, box = CASES[case]()
    e, f, w, _ = oracle.compute(pos, types, box)
    got, _ = gpu_eval(A, param_text, pos, types, box, precision=A.MIXED)
    assert_close(got, (e, f, w), 1e-6, 2e-5, 2e-5, escale="terms")


@pytest.mark.parametrize("case", ["pe1152", "hot1000"])
@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
def test_per_atom_energies(A, oracle, param_text, case, prec):
    """Per-atom energies (each term split evenly between its two atoms)
    against the oracle's, atom by atom: within 1e-10 |E| in FP64 and DF64,
    2e-6 |E| in mixed precision; through the device and the host-buffer
    calls."""
    pos, types, box = CASES[case]()
    e, _, _, _, ea = oracle.compute(pos, types, box, forces=False, per_atom=True)
    precision = {"fp64": A.FP64, "df64": A.DF64, "mixed": A.MIXED}[prec]
    tol = 2e-6 if prec == "mixed" else 1e-10
    ev = A.Airebo(param_text, precision=precision)
    p = torch.tensor(pos, device="cuda")
    ev.neighbor(p, torch.tensor(types, device="cuda"), box)
    _, e4, _, eg = ev.compute(p, per_atom=True)
    eg = eg.cpu().numpy()
    assert np.abs(eg - ea).max() <= tol * abs(e[0])
    assert abs(eg.sum() - e4[0].item()) <= 1e-12 * abs(e[0])
    ev.close()
    if prec == "fp64":
        ev = A.Airebo(param_text, precision=precision)
        _, e4h, _, eh = ev.compute_host(pos, types, box, per_atom=True)
        assert np.abs(eh - ea).max() <= tol * abs(e[0])
        ev.close()


def test_counters_match_oracle(A, oracle, param_text):
    pos, types, box = CASES["hot1000"]()
    _, _, _, c = oracle.compute(pos, types, box)
    _, ev = gpu_eval(A, param_text, pos, types, box)
    g = ev.counters()
    assert g["bonds"] == c["bonds"]
    assert g["bstar"] == c["bstar"]
    assert g["bstar_dsb"] == c["bstar_dsb_nonzero"]
    assert g["lj_in_cutoff"] == c["lj_in_cutoff"]


@pytest.mark.parametrize("case", ["pe1152", "hot160", "hot300", "hot1000", "pe32k"])
def test_bstar_screen(A, oracle, param_text, case):
    """FP64 with the b* screen (FP32 b* with a rigorous error bound, the
    default) against FP64 without it and against the oracle: the same
    energies and forces (S_b is exactly 0 or 1 wherever the screen decides),
    the bound holds on every queued pair (|b*_32 - b*_64| never exceeds it),
    and the screen leaves fewer pairs to the full pass; the 32,640-atom PE in
    full."""
    pos, types, box = CASES[case]() if case in CASES else inputs.workload(case)
    e, f, w, c = oracle.compute(pos, types, box)
    on, ev_on = gpu_eval(A, param_text, pos, types, box, bstar_screen=True)
    off, ev_off = gpu_eval(A, param_text, pos, types, box, bstar_screen=False)
    chk = ev_on.bstar_bound_check(torch.tensor(pos, device="cuda"))
    print(case, chk)
    assert chk["violations"] == 0 and chk["max_ratio"] <= 1.0
    assert chk["bounded"] + chk["unbounded"] == c["bstar"]
    # crystals: every pair bounded; hot boxes: a spline argument within its
    # bound of a knot (a bond just inside its switch) sends a pair to FP64
    assert chk["bounded"] >= (0.999 if case.startswith("pe") else 0.75) * c["bstar"]
    assert chk["max_bound"] < 1e-3
    assert_close(on, (e, f, w), 1e-10, 1e-8, 1e-8)
    assert_close(on, off, 1e-12, 1e-11, 1e-11)
    g_on, g_off = ev_on.counters(), ev_off.counters()
    assert g_on["bstar"] == g_off["bstar"] == c["bstar"]
    assert g_on["bstar_dsb"] == g_off["bstar_dsb"] == c["bstar_dsb_nonzero"]
    # without the screen the first pass decides exactly; with it, a superset
    # of the transition pairs (those within the margin) is left over
    assert g_off["bstar_full"] == g_off["bstar_dsb"]
    assert g_on["bstar_dsb"] <= g_on["bstar_full"] <= g_on["bstar"]


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("case", ["diamond216", "pe1152", "hot1000"])
def test_without_virial(A, oracle, param_text, case, precision):
    """An evaluation that asks for no virial runs the LJ kernel instance without
    virial (or parameter-gradient) accumulators: the same energies and forces
    as with the virial on the same handle, and the oracle's within the
    precision's tolerances."""
    pos, types, box = CASES[case]()
    got, ev = gpu_eval(A, param_text, pos, types, box, precision=precision, virial=False)
    p = torch.tensor(pos, device="cuda")
    f2, e2, w2 = ev.compute(p, virial=True)
    torch.cuda.synchronize()
    with_w = (e2.cpu().numpy(), f2.cpu().numpy(), w2.cpu().numpy())
    assert_close(got, with_w, 1e-12, 1e-11)
    e, f, w, _ = oracle.compute(pos, types, box)
    if precision == 1:
        assert_close(got, (e, f, w), 1e-5, 1e-4)
    else:
        assert_close(got, (e, f, w), 1e-10, 1e-8)
    ev.close()


def as_set(cnt, j, img):
    out = set()
    for i in range(len(cnt)):
        for e in range(cnt[i]):
            out.add((i, int(j[i, e]), tuple(int(s) for s in img[i, e])))
    return out


@pytest.mark.parametrize("case", ["diamond216", "hot300", "pe1152"])
def test_lists(A, oracle, params, param_text, case):
    """Index work: the exact REBO list equals the oracle's set bit for bit; the
    skin lists contain every pair within cut-off + skin (the LJ half list once,
    in one of the pair's two rows), and nothing beyond it by more than the
    FP32 margin."""
    pos, types, box = CASES[case]()
    _, ev = gpu_eval(A, param_text, pos, types, box)
    off, jj, img = oracle.rebo_neighbors(pos, types, box)
    want = {(i, int(jj[k]), tuple(int(s) for s in img[k])) for i in range(len(types)) for k in range(off[i], off[i + 1])}
    assert as_set(*ev.export_lists(2)) == want
    skin = 1.0
    for which, cut in ((0, lambda a, b: 3.0 * params["lj.sigma"][a + b]), (1, lambda a, b: params["Dmax"][a + b])):
        got = as_set(*ev.export_lists(which))
        for (i, j, S) in got:
            d = pos[:, j] + np.array(S) * box - pos[:, i]
            assert np.sqrt(d @ d) < cut(types[i], types[j]) + skin + 3e-3
            if which == 0:                  # each pair once: never also in j's row
                assert (j, i, tuple(-s for s in S)) not in got or (j == i and S > (0, 0, 0))
                assert j != i or S > (0, 0, 0)
        # every pair within cut + skin - margin is present
        rc = np.array([[cut(a, b) for b in (0, 1)] for a in (0, 1)])
        for i in range(0, len(types), 7):
            for S in np.ndindex(5, 5, 5):
                S = tuple(int(s) - 2 for s in S)
                d = pos + (np.array(S) * box)[:, None] - pos[:, i:i + 1]
                r = np.sqrt(np.einsum("ij,ij->j", d, d))
                hit = np.nonzero(r < rc[types[i], types] + skin - 3e-3)[0]
                for j in hit:
                    j = int(j)
                    if j == i and S == (0, 0, 0):
                        continue
                    if which == 1:
                        assert (i, j, S) in got
                    elif j != i or S > (0, 0, 0):      # the half list holds it in one of the two rows
                        assert (i, j, S) in got or (j, i, tuple(-s for s in S)) in got


def test_pe32k_full_parity(A, oracle, param_text):
    pos, types, box = inputs.workload("pe32k")
    e, f, w, _ = oracle.compute(pos, types, box)
    got, _ = gpu_eval(A, param_text, pos, types, box)
    assert_close(got, (e, f, w), 1e-10, 1e-8, 1e-8)
    got, _ = gpu_eval(A, param_text, pos, types, box, precision=A.MIXED)
    assert_close(got, (e, f, w), 1e-5, 1e-4, 1e-4)


def test_pe1m_sampled_parity(A, oracle, param_text):
    """The bench's 1,044,480-atom polyethylene: sampled forces against the
    oracle's one-atom-at-a-time evaluation, plus zero net force."""
    pos, types, box = inputs.workload("pe1m")
    for prec, tol in ((0, 1e-8), (A.DF64, 1e-8), (A.MIXED, 1e-4)):
        (e4, f, _), _ = gpu_eval(A, param_text, pos, types, box, precision=prec, virial=False)
        rng = np.random.default_rng(3)
        atoms = np.concatenate([[0, len(types) - 1], rng.choice(len(types), 4, replace=False)])
        if prec == 0:
            fo = oracle.forces_subset(pos, types, box, atoms)
        scale = np.abs(f).max()
        assert np.abs(f[:, atoms] - fo).max() <= tol * scale
        assert np.abs(f.sum(axis=1)).max() <= 1e-9 * scale * len(types) ** 0.5
        assert np.isfinite(e4).all() and -4.2 < e4[0] / len(types) < -3.7


def test_empty_system(A, param_text):
    ev = A.Airebo(param_text)
    p = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    ev.neighbor(p, torch.zeros(0, dtype=torch.int8, device="cuda"), [20.0, 20.0, 20.0])
    f, e4, w6 = ev.compute(p, virial=True)
    torch.cuda.synchronize()
    assert f.shape == (3, 0) and e4.abs().max().item() == 0.0 and w6.abs().max().item() == 0.0


def test_errors(A, param_text):
    ev = A.Airebo(param_text)
    pos, types, box = inputs.diamond()
    p = torch.tensor(pos, device="cuda")
    t = torch.tensor(types, device="cuda")
    with pytest.raises(A.AireboError) as ex:
        ev.compute(p)
    assert ex.value.status == A.ERR_STATE
    with pytest.raises(A.AireboError) as ex:
        ev.neighbor(p, t, [7.5, 20.0, 20.0])
    assert ex.value.status == A.ERR_ARG
    bad = p.clone()
    bad[1, 5] = float("nan")
    with pytest.raises(A.AireboError) as ex:
        ev.neighbor(bad, t, box)
    assert ex.value.status == A.ERR_NONFINITE
    ev.neighbor(p, t, box)
    with pytest.raises(A.AireboError) as ex:
        ev.compute(bad)
    assert ex.value.status == A.ERR_NONFINITE
    # two atoms at one point
    ov = p.clone()
    ov[:, 7] = ov[:, 3]
    ev.neighbor(ov, t, box)
    with pytest.raises(A.AireboError) as ex:
        ev.compute(ov)
    assert ex.value.status == A.ERR_NONFINITE and "overlapping" in str(ex.value)
    # more than 16 REBO neighbours: a cluster of 20 carbons within 2 A of each other
    rng = np.random.default_rng(0)
    cl = rng.uniform(-0.5, 0.5, (3, 20)) + 10.0
    ev2 = A.Airebo(param_text)
    pc = torch.tensor(cl, device="cuda")
    ev2.neighbor(pc, torch.zeros(20, dtype=torch.int8, device="cuda"), [20.0, 20.0, 20.0])
    with pytest.raises(A.AireboError) as ex:
        ev2.compute(pc)
    assert ex.value.status == A.ERR_CAPACITY
    with pytest.raises(A.AireboError):
        A.Airebo("not a parameter file")


def test_error_flags_reported_together(A, param_text):
    """A non-finite position and two overlapping atoms in one evaluation: both
    conditions are reported, each by its own flag bit."""
    ev = A.Airebo(param_text)
    pos, types, box = inputs.diamond()
    p = torch.tensor(pos, device="cuda")
    p[:, 7] = p[:, 3]
    ev.neighbor(p, torch.tensor(types, device="cuda"), box)
    bad = p.clone()
    bad[1, 5] = float("nan")
    with pytest.raises(A.AireboError) as ex:
        ev.compute(bad)
    assert ex.value.status == A.ERR_NONFINITE
    assert "non-finite" in str(ex.value) and "overlapping" in str(ex.value)


@pytest.mark.parametrize("precision", ["mixed", "df64"])
def test_async_check_reports_range_errors(A, param_text, precision):
    """airebo_check after an asynchronous evaluation returns the errors the
    synchronous call returns: a coordinate beyond 2000 A on the split positions
    of the mixed and DF64 paths."""
    pos, types, box = CASES["pe1152"]()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ev = A.Airebo(param_text, precision=A.MIXED if precision == "mixed" else A.DF64, stream=stream)
        p = torch.tensor(pos + 2100.0, device="cuda")
        ev.neighbor(p, torch.tensor(types, device="cuda"), box)
        f = torch.empty_like(p)
        ev.compute_async(p, f)
        with pytest.raises(A.AireboError) as ex:
            ev.check()
        assert ex.value.status == A.ERR_ARG and "2000" in str(ex.value)
        # and a clean evaluation afterwards checks clean
        q = torch.tensor(pos, device="cuda")
        ev.neighbor(q, torch.tensor(types, device="cuda"), box)
        ev.compute(q)
        ev.compute_async(q, f)
        ev.check()
        ev.close()


def test_capacity_regrow(A, oracle, param_text):
    """A long-list capacity far too small is grown, and the result is exact."""
    pos, types, box = CASES["hot300"]()
    e, f, w, _ = oracle.compute(pos, types, box)
    got, ev = gpu_eval(A, param_text, pos, types, box, max_lj_nbrs=8)
    assert ev.counters()["lj_cap"] > 8
    assert_close(got, (e, f, w), 1e-10, 1e-8, 1e-8)


def test_host_api_matches_device(A, param_text):
    pos, types, box = CASES["hot300"]()
    (e4, f, w), _ = gpu_eval(A, param_text, pos, types, box)
    ev = A.Airebo(param_text)
    fh, eh, wh = ev.compute_host(pos, types, box, virial=True)
    assert np.abs(fh - f).max() <= 1e-12 * np.abs(f).max()
    assert abs(eh[0] - e4[0]) <= 1e-12 * abs(e4[0])


def oracle_nve(oracle, pos, vel, types, box, dt, nsteps):
    m = inputs.masses(types)
    e, f, _, _ = oracle.compute(pos, types, box)
    x, v = pos.copy(), vel.copy()
    for _ in range(nsteps):
        v += 0.5 * dt * f / m / inputs.MVV2E
        x += dt * v
        e, f, _, _ = oracle.compute(x, types, box)
        v += 0.5 * dt * f / m / inputs.MVV2E
    ke = 0.5 * inputs.MVV2E * (m * v * v).sum()
    return x, v, e[0], ke


@pytest.mark.parametrize("case,temp,precision,xtol,etol", [
    ("hot300", 2000.0, 0, 1e-8, 1e-9),
    ("pe1152", 600.0, 0, 1e-8, 1e-9),
    ("pe1152", 600.0, 2, 1e-8, 1e-9),
    ("pe1152", 600.0, 1, 1e-4, 1e-5),
])
def test_nve_against_oracle_trajectory(A, oracle, param_text, case, temp, precision, xtol, etol):
    """Velocity Verlet on the GPU follows the oracle-driven trajectory, with
    list rebuilds on the way (small skin).  The mixed path is checked on PE:
    on the hot reactive box a near-tie in the C_ij argmax flips in FP32 and
    the chaotic trajectory separates, as any reduced-precision run would."""
    pos, types, box = CASES[case]()
    vel = inputs.velocities(types, temp, seed=4)
    x_o, v_o, pe_o, ke_o = oracle_nve(oracle, pos, vel, types, box, 0.5, 20)
    ev = A.Airebo(param_text, precision=precision, skin=0.15)
    p = torch.tensor(pos, device="cuda")
    v = torch.tensor(vel, device="cuda")
    ev.neighbor(p, torch.tensor(types, device="cuda"), box)
    f, _, _ = ev.compute(p)
    e4 = ev.nve(p, v, f, 0.5, 20).cpu().numpy()
    assert e4[3] > 1                      # the lists were rebuilt on the way
    assert np.abs(p.cpu().numpy() - x_o).max() < xtol
    assert abs(e4[0] - pe_o) <= etol * abs(pe_o)
    assert abs(e4[1] - ke_o) <= etol * 10 * abs(ke_o)


@pytest.mark.parametrize("precision", [0, 2])
def test_trace_rerun_frames(A, oracle, param_text, precision):
    """Trace dump and rerun: the oracle drives a hot reactive NVE run (2000 K,
    bonds forming and breaking) and records 20 frames; the GPU path then
    evaluates every recorded frame on its own, so both see identical inputs,
    and each frame's energy and forces must match the oracle's."""
    pos, types, box = CASES["hot300"]()
    vel = inputs.velocities(types, 2000.0, seed=9)
    m = np.where(types == 0, 12.011, 1.008)
    dt = 0.5
    x, v = pos.copy(), vel.copy()
    e, f, _, _ = oracle.compute(x, types, box)
    frames = []
    for _ in range(20):
        v += 0.5 * dt * f / m / inputs.MVV2E
        x += dt * v
        e, f, _, _ = oracle.compute(x, types, box)
        v += 0.5 * dt * f / m / inputs.MVV2E
        frames.append((x.copy(), e.copy(), f.copy()))
    ev = A.Airebo(param_text, precision=precision, skin=0.1)
    t = torch.tensor(types, device="cuda")
    for k, (xk, ek, fk) in enumerate(frames):
        p = torch.tensor(xk, device="cuda")
        ev.neighbor(p, t, box)
        fg, eg, _ = ev.compute(p)
        torch.cuda.synchronize()
        eg = eg.cpu().numpy()
        fg = fg.cpu().numpy()
        assert abs(eg[0] - ek[0]) <= 1e-10 * abs(ek[0]), (k, eg, ek)
        assert np.abs(fg - fk).max() <= 1e-8 * np.abs(fk).max(), (k, np.abs(fg - fk).max())
    ev.close()


def test_nve_resume_from_checkpoint(A, param_text, tmp_path):
    """Ten NVE steps in one run equal five steps, a checkpoint file, and five
    more steps on a fresh handle built from the file (to the order of the
    atomic sums)."""
    from paper_1810_07026_gb300 import checkpoint
    pos, types, box = CASES["pe1152"]()
    vel = inputs.velocities(types, 600.0, seed=6)
    t = torch.tensor(types, device="cuda")

    def run(p0, v0, steps):
        ev = A.Airebo(param_text)
        p = torch.tensor(p0, device="cuda")
        v = torch.tensor(v0, device="cuda")
        ev.neighbor(p, t, box)
        f, _, _ = ev.compute(p)
        e4 = ev.nve(p, v, f, 0.5, steps)
        torch.cuda.synchronize()
        ev.close()
        return p.cpu().numpy(), v.cpu().numpy(), e4.cpu().numpy()

    x10, v10, e10 = run(pos, vel, 10)
    x5, v5, _ = run(pos, vel, 5)
    f = tmp_path / "md.npz"
    checkpoint.save(str(f), x5, v5, types, box, 5, dt=0.5, precision=A.FP64, skin=1.0, params=param_text)
    s = checkpoint.load(str(f))
    assert s["step"] == 5
    checkpoint.check_evaluator(s, A.Airebo(s["params"], precision=s["precision"], skin=s["skin"]), dt=0.5)
    with pytest.raises(ValueError):
        checkpoint.check_evaluator(s, A.Airebo(param_text, precision=A.MIXED), dt=0.5)
    xr, vr, er = run(s["pos"], s["vel"], 5)
    assert np.abs(xr - x10).max() < 1e-10
    assert np.abs(vr - v10).max() < 1e-10
    assert abs(er[2] - e10[2]) <= 1e-10 * abs(e10[2])


def test_nve_energy_conservation(A, param_text):
    pos, types, box = inputs.diamond()
    vel = inputs.velocities(types, 1000.0, seed=3)
    ev = A.Airebo(param_text)
    p = torch.tensor(pos, device="cuda")
    v = torch.tensor(vel, device="cuda")
    ev.neighbor(p, torch.tensor(types, device="cuda"), box)
    f, _, _ = ev.compute(p)
    tot = []
    for _ in range(20):
        tot.append(ev.nve(p, v, f, 0.5, 5)[2].item())
    tot = np.array(tot)
    assert (tot.max() - tot.min()) < 3e-4 * abs(tot[0])


@pytest.mark.parametrize("precision", [0, 1])
def test_nve_pe32k_1000_steps_energy(A, param_text, precision):
    """1,000 velocity-Verlet steps of 0.5 fs on the 32,640-atom PE at 300 K:
    the total energy fluctuates (Verlet) but does not drift."""
    pos, types, box = inputs.workload("pe32k")
    vel = inputs.velocities(types, 300.0, seed=2)
    n = len(types)
    ev = A.Airebo(param_text, precision=precision)
    p = torch.tensor(pos, device="cuda")
    v = torch.tensor(vel, device="cuda")
    ev.neighbor(p, torch.tensor(types, device="cuda"), box)
    f, _, _ = ev.compute(p)
    tot = []
    for _ in range(20):
        e4 = ev.nve(p, v, f, 0.5, 50).cpu().numpy()
        tot.append(e4[2] / n)
    tot = np.array(tot)
    slope = np.polyfit(np.arange(len(tot)) * 50.0, tot, 1)[0]        # eV/atom/step
    print(f"precision {precision}: E/atom spread {tot.max() - tot.min():.3e}, drift {slope:.3e} eV/atom/step, "
          f"list builds {e4[3]:.0f}")
    assert tot.max() - tot.min() < 2e-3
    assert abs(slope) < 5e-7


@pytest.mark.parametrize("case", ["hot300", "pe1152", "diamond216"])
@pytest.mark.parametrize("precision,etol,ftol", [(0, 1e-10, 1e-8), (1, 1e-5, 1e-4), (2, 1e-10, 1e-8)])
def test_morse_parity(A, case, precision, etol, ftol):
    """AIREBO-M: the Morse inter-molecular term, GPU against the oracle (with
    the Morse form DF64 and mixed run their LJ pairs without the split)."""
    from oracle.oracle import Oracle
    text = inputs.params_text(inputs.make_params(0, morse=True))
    pos, types, box = CASES[case]()
    e, f, w, _ = Oracle(text).compute(pos, types, box)
    got, _ = gpu_eval(A, text, pos, types, box, precision=precision)
    assert_close(got, (e, f, w), etol, ftol, ftol)
