#!/usr/bin/env python
"""AIREBO MD throughput on one GB300: atom-steps/s on 1,044,480-atom polyethylene.

A step is one velocity-Verlet NVE step of the whole hot path: half kick and
drift, the displacement check that triggers a list rebuild (binning, LJ half
list, REBO intermediate list) when an atom moved more than skin/2, the exact
REBO list, REBO bonds with the bond order, torsion, the connectivity map, the
LJ pairs, the deferred b* pairs, and the second half kick.  `value` is the
FP64 path (every term in FP64; S_b of a b* pair is decided from an FP32 b*
only where its rigorous error bound puts it outside the S_b transition, and
every other b* is FP64); the mixed path (FP32 geometry/splines/bond order,
FP64 accumulation), the DF64 path and the FP64 path without the b* screen
are reported beside it with their max |dF| against FP64.  The energy drift of the FP64 and mixed paths is the
least-squares slope of the total energy over 200 NVE steps after the timed
region, at the bench's dt = 0.5 fs and again from the same state at 0.25 fs
(a few hydrogen atoms of this noisy start run hot, and their close collisions
need the shorter step).

Timing: W untimed warm-up steps, then K steps bracketed by a barrier and
torch.cuda.synchronize(), timed with CUDA events on the library's stream; the
working set (~3 GB of lists, 50 MB of positions and forces) is larger than the
L2, so no flush is needed.  Per-kernel times come from CUDA events the library
records around each launch during the same timed region.

--impl reference times the plain FP64 CPU oracle on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1810_07026_gb300 import inputs  # noqa: E402

METRIC = "AIREBO atom-steps/s (1M-atom PE) FP64 vs mixed on GB300; max |dF| vs FP64 oracle"
UNIT = "atom-steps/s"
WORKLOAD = "pe1m"
DT = 0.5
TEMP = 300.0
DRIFT_STEPS = 200         # NVE steps after the timed region whose total energy is fitted for the drift

# Algorithmic FP64 work per unit, in flops (FMA = 2).
FLOPS_LJ_PAIR = 44        # displacement with image (9), r^2 (5), sqrt, 1/r, (s/r)^6, V, dV/dr, force, sums (30)
FLOPS_LJ_TEST = 14        # displacement and r^2 of a pair that is tested but not evaluated (C = 0, or queued for b*)
# DRAM bytes (read + write) per atom of one k_lj<double> launch and the
# k_lj_path launch that follows it (the LJ stage the bench times), measured by
# ncu (dram__bytes_read.sum + dram__bytes_write.sum) on the 261,120-atom PE
# with the same kernels: 724.4 + 21.6 MB and 9.0 + 0.1 MB per launch.  The
# traffic is the list read and the connectivity-map probes, whose size per
# atom the density fixes, so it scales with the atom count.
LJ_DRAM_BYTES_PER_ATOM = (724.409856e6 + 21.606144e6 + 8.958208e6 + 0.11776e6) / 261120
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP64_FMA_PER_SM_CLK = 2   # 1.25 TFLOP/s nominal FP64 = 152 SMs x 2 FMA x 2 flop x 2.07 GHz
FP32_FMA_PER_SM_CLK = 128


def hbm_peak():
    """HBM bandwidth in GB/s: the measured copy rate of these GPUs when the
    measurement file sits beside this script, else an earlier measurement."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def peaks_nominal():
    f64 = SM_COUNT * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
    f32 = SM_COUNT * FP32_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
    return f64, f32


def max_over_ranks(value: float, dist, device) -> float:
    """The largest of the ranks' values (the slowest rank's time); the value
    itself when there is no process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(n_atoms: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job atom-steps/s of `world` independent replicas (weak scaling)."""
    return world * n_atoms * steps / (max_ms * 1e-3)


def config_of(workload: str, n: int, world: int) -> dict:
    return {"workload": f"polyethylene {workload}: {n} atoms, 300 K, dt 0.5 fs, skin 1 A",
            "global_batch": n * world, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "working set > L2 (lists ~3 GB at 1M atoms), no flush"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"airebo_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip() + f", {os.cpu_count()} logical CPUs"
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def oracle_sample(pos, types, box, target_s, threads=None):
    """Time the CPU oracle on a sphere of anchor atoms of the workload, sized
    to take about target_s seconds.  Returns (atom-steps/s, threads, sample text, counters per anchor)."""
    from oracle import oracle as O
    if threads:
        O.set_threads(threads)
    o = O.Oracle(inputs.params_text(inputs.make_params(0)))
    center = int(np.argmin(np.abs(pos - (box / 2)[:, None]).sum(axis=0)))
    r = 20.0
    for _ in range(5):
        t0 = time.perf_counter()
        _, _, c, na = o.evaluate_sphere(pos, types, box, center, r)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * target_s:
            break
        r *= min(2.0, (target_s / max(dt, 1e-3)) ** (1.0 / 3.0))
    nth = O.threads()
    per = {k: v / na for k, v in c.items()}
    sample = f"all terms anchored at the {na} atoms within {r:.1f} A of the box centre of the 1,044,480-atom PE, one force evaluation"
    return na / dt, nth, sample, per, dt


def drift_fit(etot, n_atoms):
    """Least-squares slope of the total energy per atom over consecutive NVE
    steps (eV/atom/step) and its spread (max - min, eV/atom)."""
    e = np.asarray(etot, dtype=np.float64) / n_atoms
    k = np.arange(len(e), dtype=np.float64)
    slope = float(np.polyfit(k, e, 1)[0]) if len(e) > 1 else 0.0
    return {"slope_eV_per_atom_step": slope, "spread_eV_per_atom": float(e.max() - e.min()), "steps": len(e),
            "method": "least-squares slope of E_total/N over consecutive NVE steps after the timed region"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    pos, types, box = inputs.workload(args.workload)
    rates = []
    nth = None
    sample = ""
    for k in range(args.warmup + args.steps):
        target = max(2.0, min(8.0, 150.0 / max(1, args.warmup + args.steps)))
        rate, nth, sample, _, _ = oracle_sample(pos, types, box, target)
        if k >= args.warmup:
            rates.append(rate)
    v = float(np.median(rates))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * len(types) / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args.workload, len(types), 1),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": nth, "kind": "oracle",
                             "sample": sample + " per step; value is the median over the steps",
                             "cpu": cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args, A, params, dev, stream):
    """256 independent amorphous C:H boxes (200-8,000 atoms, H/C 0.5-2, 0.9 g/cm^3),
    relaxed by 200 FP64 steepest-descent steps (untimed), then evaluated in mixed
    precision: one captured CUDA graph for all systems against a loop over one
    handle per system."""
    import torch
    from paper_1810_07026_gb300 import batch
    P, T, O, B = inputs.ensemble(256)
    nat = int(O[-1])
    pos = torch.tensor(P, device=dev)
    typ = torch.tensor(T, device=dev)
    batch.relax(params, pos, typ, O, B, steps=200)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ev = A.Airebo(params, precision=A.MIXED, stream=stream)
        ev.neighbor_batch(pos, typ, O, B)
        f = torch.zeros_like(pos)
        e = torch.zeros(len(B), dtype=torch.float64, device=dev)
        ev.graph_capture(pos, f, None, e)
        for _ in range(args.warmup):
            ev.graph_launch()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            ev.graph_launch()
        e1.record(stream)
        e1.synchronize()
        ev.check()
        ms_graph = e0.elapsed_time(e1) / args.steps
        ev.close()
        hs, ps = [], []
        for s in range(len(B)):
            h = A.Airebo(params, precision=A.MIXED, stream=stream)
            p = pos[:, O[s]:O[s + 1]].contiguous()
            h.neighbor(p, typ[O[s]:O[s + 1]].contiguous(), B[s])
            hs.append(h); ps.append(p)
        for h, p in zip(hs, ps):
            h.compute(p)
        stream.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            for h, p in zip(hs, ps):
                h.compute(p)
        e1.record(stream)
        e1.synchronize()
        ms_loop = e0.elapsed_time(e1) / args.steps
        # MD: K velocity-Verlet steps of every system (rebuilds decided on the
        # device) in one graph launch, against K airebo_nve steps of each
        # per-system handle in turn (the host decides each rebuild)
        K = 10
        vel0 = inputs.velocities(T, 300.0, seed=3)
        md = A.Airebo(params, precision=A.MIXED, stream=stream)
        pm = pos.clone()
        vm = torch.tensor(vel0, device=dev)
        md.neighbor_batch(pm, typ, O, B)
        fm = torch.zeros_like(pm)
        reps = max(1, args.steps // 5)
        recaptures = 0
        p_init, v_init = pm.clone(), vm.clone()
        for attempt in range(3):
            # a capacity exceeded during the replays: start again from the
            # first state with a new capture (which grows every capacity)
            pm.copy_(p_init)
            vm.copy_(v_init)
            md.graph_capture_nve(pm, vm, fm, DT, K)
            md.graph_launch()
            try:
                md.check()
            except A.AireboError as ex:
                if ex.status != A.ERR_CAPACITY:
                    raise
                recaptures += 1
                continue
            stream.synchronize()
            e0.record(stream)
            for _ in range(reps):
                md.graph_launch()
            e1.record(stream)
            e1.synchronize()
            try:
                md.check()
            except A.AireboError as ex:
                if ex.status != A.ERR_CAPACITY:
                    raise
                recaptures += 1
                continue
            break
        ms_md_graph = e0.elapsed_time(e1) / (reps * K)
        md.close()
        vs = [torch.tensor(vel0[:, O[s]:O[s + 1]], device=dev) for s in range(len(B))]
        fs = []
        for h, p in zip(hs, ps):
            fs.append(h.compute(p)[0])
        for h, p, v, f in zip(hs, ps, vs, fs):
            h.nve(p, v, f, DT, 1)
        stream.synchronize()
        e0.record(stream)
        for h, p, v, f in zip(hs, ps, vs, fs):
            h.nve(p, v, f, DT, K)
        e1.record(stream)
        e1.synchronize()
        ms_md_loop = e0.elapsed_time(e1) / K
        for h in hs:
            h.close()
    return {"systems": len(B), "atoms": nat, "dtype": "mixed", "unit": "atom-evaluations/s",
            "graph": nat / (ms_graph * 1e-3), "graph_ms": ms_graph,
            "loop": nat / (ms_loop * 1e-3), "loop_ms": ms_loop, "speedup": ms_loop / ms_graph,
            "md": {"unit": "atom-steps/s", "steps_per_graph_launch": K, "recaptures": recaptures,
                   "graph": nat / (ms_md_graph * 1e-3), "graph_ms_per_step": ms_md_graph,
                   "loop": nat / (ms_md_loop * 1e-3), "loop_ms_per_step": ms_md_loop,
                   "speedup": ms_md_loop / ms_md_graph,
                   "what": "velocity-Verlet steps (dt 0.5 fs, 300 K) of all systems, list rebuilds decided on the "
                           "device, as one CUDA graph of 10 steps; loop: airebo_nve on each system's own handle"},
            "workload": "amorphous C:H boxes 200-8000 atoms, H/C 0.5-2.0, 0.9 g/cm^3, relaxed 200 SD steps"}


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    from paper_1810_07026_gb300 import build, airebo
    build.build()
    A = airebo
    params = inputs.params_text(inputs.make_params(0))
    pos0, types, box = inputs.workload(args.workload)
    vel0 = inputs.velocities(types, TEMP, seed=2)
    n = len(types)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream()
    results = {}
    forces = {}
    # name, precision, all terms, b* screen (FP32 b* with a rigorous error bound; the
    # default; the run without it evaluates every b* in FP64)
    runs = ((A.FP64, "fp64", True, True), (A.FP64, "fp64_no_bstar_screen", True, False), (A.MIXED, "mixed", True, True),
            (A.DF64, "df64", True, True), (A.FP64, "rebo_only", False, True))
    for prec, name, full, screen in runs:
        with torch.cuda.stream(stream):
            ev = A.Airebo(params, precision=prec, stream=stream, lj=full, torsion=full, bstar_screen=screen)
            pos = torch.tensor(pos0, device=dev)
            vel = torch.tensor(vel0, device=dev)
            t = torch.tensor(types, device=dev)
            ev.neighbor(pos, t, box)
            shape = ev.autotune(pos)
            f, e4, _ = ev.compute(pos)
            forces[name] = f.clone()
            ev.nve(pos, vel, f, DT, 1)
            for _ in range(max(0, args.warmup - 1)):
                ev.nve(pos, vel, f, DT, 1)
            builds0 = ev.counters()["list_builds"]
            stream.synchronize()
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            clocks = Clocks(local) if name == "fp64" else None
            if clocks:
                clocks.start()
            ev.set_timing(True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                ev.nve(pos, vel, f, DT, 1)
            e1.record(stream)
            e1.synchronize()
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            ck = clocks.stop() if clocks else None
            kt = ev.kernel_times()
            ev.set_timing(False)
            builds = ev.counters()["list_builds"] - builds0
            counters = ev.counters()
            drift = None
            if name in ("fp64", "mixed") and args.drift_steps > 1:
                # from the state after the timed steps: dt = 0.5 fs (the bench's step),
                # then again from that state at dt = 0.25 fs
                p0, v0 = pos.clone(), vel.clone()
                drift = {}
                mass = torch.tensor(inputs.masses(types), device=dev)
                for dt in (DT, 0.5 * DT):
                    pos.copy_(p0)
                    vel.copy_(v0)
                    ev.neighbor(pos, t, box)
                    ev.compute(pos, f)
                    etot = [ev.nve(pos, vel, f, dt, 1)[2].clone() for _ in range(args.drift_steps)]
                    fit = drift_fit(torch.stack(etot).cpu().numpy(), n)
                    fit["hottest_atom_KE_eV"] = float((0.5 * inputs.MVV2E * (mass * vel * vel).sum(0)).max().item())
                    drift[f"dt_{dt:g}fs"] = fit
            ms = max_over_ranks(ms, dist, dev)
            results[name] = dict(ms=ms, kt=kt, clocks=ck, shape=shape, builds=builds, counters=counters,
                                 drift=drift)
            ev.close()
    # mixed against FP64 at the same (initial) positions
    df = (forces["mixed"] - forces["fp64"]).abs().max().item()
    fscale = forces["fp64"].abs().max().item()

    # e2e through the host-buffer API (FP64): copy in, one step, copy out, every step
    e2e = None
    with torch.cuda.stream(stream):
        ev = A.Airebo(params, precision=A.FP64, stream=stream)
        ev.set_launch_shape(*results["fp64"]["shape"])
        hp = torch.tensor(pos0).pin_memory()
        hv = torch.tensor(vel0).pin_memory()
        hf = torch.zeros_like(hp).pin_memory()
        fh, _, _ = ev.compute_host(hp.numpy(), types, box)
        hf.copy_(torch.from_numpy(fh))
        for _ in range(args.warmup):
            ev.nve_host(hp, hv, hf, DT, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ev.nve_host(hp, hv, hf, DT, 1)
        dt_e2e = time.perf_counter() - t0
        ev.close()
        e2e = {"value": n * args.steps / dt_e2e, "unit": UNIT, "h2d_bytes_per_step": 3 * 24 * n,
               "d2h_bytes_per_step": 3 * 24 * n + 32}

    batched = run_batched(args, A, params, dev, stream) if args.batch else None

    r64 = results["fp64"]
    value = replica_throughput(n, args.steps, ws, r64["ms"])
    mixed_value = replica_throughput(n, args.steps, ws, results["mixed"]["ms"])
    # roofline of the dominant kernel (FP64 path)
    kt = r64["kt"]
    dom = max((k for k in kt if k not in ("neighbor",)), key=lambda k: kt[k][0])
    peak64_nom, peak32_nom = peaks_nominal()
    peak64_meas = A.alu_peak(A.FP64)
    peak32_meas = A.alu_peak(A.MIXED)

    line = None
    if rank == 0:
        # algorithmic work from the oracle's term counters on a bounded sample
        cpu_rate, nth, sample, per, cpu_dt = oracle_sample(pos0, types, box, target_s=12.0)
        cpu1_rate, _, sample1, _, cpu1_dt = oracle_sample(pos0, types, box, target_s=4.0, threads=1)
        from oracle import oracle as O
        O.set_threads(nth)
        pairs_eval = per["lj_in_cutoff"] - per["lj_c_zero"] - per["bstar"]
        pairs_test = per["lj_c_zero"] + per["bstar"]
        flops_lj = n * (FLOPS_LJ_PAIR * pairs_eval + FLOPS_LJ_TEST * pairs_test)
        lj_ms, lj_n = kt["lj"]
        lj_avg_s = lj_ms * 1e-3 / max(1, lj_n)
        achieved = flops_lj / lj_avg_s / 1e12 if dom == "lj" else None
        mix_kt = results["mixed"]["kt"]
        mlj_ms, mlj_n = mix_kt["lj"]
        roof = {"kernel": "k_lj<double>", "bound": "alu", "achieved": achieved, "peak": peak64_nom,
                "unit": "TFLOP/s", "frac": (achieved / peak64_nom) if achieved else None,
                "traffic": LJ_DRAM_BYTES_PER_ATOM * n if args.workload.startswith("pe") else None,
                "traffic_unit": "bytes per k_lj + k_lj_path launch pair (ncu, 261,120-atom PE, scaled by atoms)",
                "peak_kind": "FP64 nominal from SM count x FMA units x max clock; measured FMA probe beside it",
                "peak_measured": peak64_meas,
                "flops_per_launch": flops_lj, "avg_launch_ms": lj_avg_s * 1e3,
                "dominant_kernel": dom}
        if roof["traffic"]:
            hbm, hbm_kind = hbm_peak()
            gbs = roof["traffic"] / lj_avg_s / 1e9
            roof["hbm"] = {"achieved_gbs": gbs, "peak_gbs": hbm, "peak_kind": hbm_kind, "frac": gbs / hbm}
        # per timed step (one airebo_nve call): two half-step kernels, the ten
        # kernels of an evaluation (FP32 positions, short list, REBO, torsion,
        # map, LJ, LJ pairs along a path, two b* passes, counters) and the
        # energy write; five more per list rebuild (bin, scan, scatter, build,
        # order)
        launches = 13 * args.steps + 5 * r64["builds"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r64["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args.workload, n, ws),
            "mixed": {"value": mixed_value, "unit": UNIT, "ms_per_step": results["mixed"]["ms"] / args.steps,
                      "max_abs_dF_vs_fp64": df, "max_rel_dF_vs_fp64": df / fscale,
                      "drift": results["mixed"]["drift"],
                      "kernel_ms": {k: v[0] / max(1, v[1]) for k, v in mix_kt.items()},
                      "lj_achieved_fp32_frac": None if not mlj_n else
                      (flops_lj / (mlj_ms * 1e-3 / mlj_n) / 1e12) / peak32_nom},
            "df64": {"value": replica_throughput(n, args.steps, ws, results["df64"]["ms"]), "unit": UNIT,
                     "ms_per_step": results["df64"]["ms"] / args.steps,
                     "dtype": "f64; LJ pair and torsion arithmetic in double-float (f32 pairs), LJ forces in 64-bit fixed point",
                     "max_abs_dF_vs_fp64": (forces["df64"] - forces["fp64"]).abs().max().item(),
                     "max_rel_dF_vs_fp64": (forces["df64"] - forces["fp64"]).abs().max().item() / fscale,
                     "kernel_ms": {k: v[0] / max(1, v[1]) for k, v in results["df64"]["kt"].items()}},
            "fp64_no_bstar_screen": {
                "value": replica_throughput(n, args.steps, ws, results["fp64_no_bstar_screen"]["ms"]), "unit": UNIT,
                "ms_per_step": results["fp64_no_bstar_screen"]["ms"] / args.steps,
                "dtype": "f64, every b* evaluated in FP64 (no screen)",
                "max_abs_dF_vs_fp64": (forces["fp64_no_bstar_screen"] - forces["fp64"]).abs().max().item(),
                "kernel_ms": {k: v[0] / max(1, v[1]) for k, v in results["fp64_no_bstar_screen"]["kt"].items()}},
            "batched": batched,
            "rebo_only": {"value": replica_throughput(n, args.steps, ws, results["rebo_only"]["ms"]),
                          "unit": UNIT, "ms_per_step": results["rebo_only"]["ms"] / args.steps,
                          "dtype": "f64", "terms": "REBO (Alg. 1) only, no LJ or torsion, no long list",
                          "kernel_ms": {k: v[0] / max(1, v[1]) for k, v in results["rebo_only"]["kt"].items()}},
            "drift": r64["drift"],
            "list_builds_in_timed_region": r64["builds"],
            "launch_shape": {k: {"lj_atoms_per_claim": results[k]["shape"][0],
                                 "bond_waves": results[k]["shape"][1],
                                 "bstar_waves": results[k]["shape"][2]} for k in results},
            "kernel_ms": {k: v[0] / max(1, v[1]) for k, v in kt.items()},
            "kernel_share": {k: v[0] / max(1e-9, sum(x[0] for x in kt.values())) for k, v in kt.items()},
            "roofline": roof,
            "peaks_TFLOPs": {"fp64_nominal": peak64_nom, "fp64_measured": peak64_meas,
                             "fp32_nominal": peak32_nom, "fp32_measured": peak32_meas},
            "cpu_baseline": {"value": cpu_rate, "unit": UNIT, "cores": nth, "kind": "oracle", "sample": sample,
                             "cpu": cpu_model(), "seconds": cpu_dt,
                             "single_thread": {"value": cpu1_rate, "cores": 1, "sample": sample1,
                                               "seconds": cpu1_dt}},
            "counters_fp64_last_step": {k: v for k, v in r64["counters"].items() if k != "list_builds"},
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": r64["clocks"],
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-batch", dest="batch", action="store_false",
                    help="leave out the batched-ensemble comparison (profiler captures)")
    ap.add_argument("--drift-steps", dest="drift_steps", type=int, default=DRIFT_STEPS,
                    help="NVE steps after the timed region whose energy slope is reported (FP64 and mixed)")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(inputs.WORKLOADS),
                    help="pe1m is the benchmark; the smaller ones exist for profiler captures")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
