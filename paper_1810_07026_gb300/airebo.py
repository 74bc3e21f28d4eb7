"""Python binding of libairebo (ctypes): argument marshalling only.

Every step of the evaluation runs in the CUDA library declared in
``include/airebo.h``; this module passes torch device pointers and the
current CUDA stream through.  It raises if the library is missing -- there is
no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import inputs

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libairebo.so")

OK, ERR_ARG, ERR_CUDA, ERR_CAPACITY, ERR_TIMEOUT, ERR_NONFINITE, ERR_STATE = range(7)
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_CAPACITY", 4: "ERR_TIMEOUT", 5: "ERR_NONFINITE", 6: "ERR_STATE"}
FP64, MIXED, DF64 = 0, 1, 2
# the spline knot data, in the order of the parameter file and of knot_grad()
KNOT_BLOCKS = (("gC1.data", 18), ("gC2.data", 18), ("gH.data", 12), ("P.CC", 100), ("P.CH", 100), ("P.HC", 100),
               ("piRC.CC", 1800), ("piRC.CH", 1800), ("piRC.HH", 1800), ("Tij.CC", 1800))
KNOT_COUNT = sum(c for _, c in KNOT_BLOCKS)
KERNELS = ("short_list", "rebo", "torsion", "path_map", "lj", "bstar", "neighbor", "nve", "bstar_rev")


class AireboError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [("skin", C.c_double), ("precision", C.c_int), ("enable_rebo", C.c_int),
                ("enable_lj", C.c_int), ("enable_torsion", C.c_int), ("max_lj_nbrs", C.c_int),
                ("bstar_screen", C.c_int)]


_lib = None


def lib():
    """The loaded libairebo.so; raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libairebo.so is not built ({LIB_PATH}); run paper_1810_07026_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        P, I64, D, I = C.c_void_p, C.c_int64, C.c_double, C.c_int
        sig = {
            "airebo_default_options": (None, [P]),
            "airebo_create": (I, [C.c_char_p, P, P, P]),
            "airebo_destroy": (None, [P]),
            "airebo_last_error": (C.c_char_p, [P]),
            "airebo_neighbor": (I, [P, P, P, I64, P]),
            "airebo_compute": (I, [P, P, P, P, P, P]),
            "airebo_compute_host": (I, [P, P, P, I64, P, P, P, P, P]),
            "airebo_needs_rebuild": (I, [P, P, P]),
            "airebo_nve": (I, [P, P, P, P, D, I, P]),
            "airebo_nve_host": (I, [P, P, P, P, D, I, P]),
            "airebo_counters": (I, [P, P]),
            "airebo_export_lists": (I, [P, I, P, P, P, I64]),
            "airebo_set_timing": (I, [P, I]),
            "airebo_kernel_times": (I, [P, P, P]),
            "airebo_alu_peak": (I, [I, P]),
            "airebo_math_check": (I, [P]),
            "airebo_dd_check": (I, [P]),
            "airebo_param_grad": (I, [P, P, P, P, P]),
            "airebo_knot_grad": (I, [P, P, P, P, P, I64]),
            "airebo_set_lj_params": (I, [P, P, P]),
            "airebo_neighbor_batch": (I, [P, P, P, I64, I, P, P]),
            "airebo_compute_batch": (I, [P, P, P, P]),
            "airebo_compute_async": (I, [P, P, P, P, P]),
            "airebo_check": (I, [P]),
            "airebo_graph_capture": (I, [P, P, P, P, P]),
            "airebo_graph_launch": (I, [P]),
            "airebo_autotune": (I, [P, P, P, P]),
            "airebo_set_launch_shape": (I, [P, I, I, I]),
            "airebo_set_knots": (I, [P, P, I64]),
            "airebo_nve_async": (I, [P, P, P, P, D, I, P]),
            "airebo_force_param_grad": (I, [P, P, P, P, P, P]),
            "airebo_bstar_bound_check": (I, [P, P, P, P]),
            "airebo_graph_capture_nve": (I, [P, P, P, P, D, I, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _np(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def alu_peak(precision: int = FP64) -> float:
    """Measured FMA TFLOP/s of the current device (FP64 or FP32)."""
    out = C.c_double(0)
    st = lib().airebo_alu_peak(precision, C.byref(out))
    if st:
        raise AireboError(st, "alu peak probe failed")
    return out.value


def dd_check():
    """Largest errors of the double-float operations (add relative to |a|+|b|; mul, div, rcp, rsqrt
    relative; sin(pi t), cos(pi t) absolute; conversion from double relative)."""
    out = np.zeros(8, dtype=np.float64)
    st = lib().airebo_dd_check(_np(out))
    if st:
        raise AireboError(st, "double-float check failed")
    return dict(zip(("add", "mul", "div", "rcp", "rsqrt", "sinpi", "cospi", "from_double"), out.tolist()))


def math_check():
    """ulp differences from CUDA's correctly rounded results: the kernels' 1/x and 1/sqrt(x), then
    the hardware approximations alone."""
    out = np.zeros(4, dtype=np.int64)
    st = lib().airebo_math_check(_np(out))
    if st:
        raise AireboError(st, "math check failed")
    return tuple(int(v) for v in out)


class Airebo:
    """One AIREBO evaluator on the current CUDA device and stream.

    Positions, forces and velocities are torch float64 tensors of shape
    (3, N) on the device (structure of arrays), types int8 (N,)."""

    def __init__(self, params: str | dict | None = None, precision: int = FP64, skin: float = 1.0,
                 rebo: bool = True, lj: bool = True, torsion: bool = True, max_lj_nbrs: int = 0, stream=None,
                 bstar_screen: bool = True):
        import torch
        self._torch = torch
        if params is None:
            params = inputs.make_params(0)
        if isinstance(params, dict):
            params = inputs.params_text(params)
        opt = Options(skin, precision, int(rebo), int(lj), int(torsion), int(max_lj_nbrs), int(bstar_screen))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.device = stream.device
        h = C.c_void_p()
        st = lib().airebo_create(params.encode(), C.byref(opt), C.c_void_p(stream.cuda_stream), C.byref(h))
        if st:
            raise AireboError(st, "airebo_create failed")
        self._h = h
        self.n = None
        self.precision = precision
        self.skin = float(skin)
        self.params_text = params

    def close(self):
        if getattr(self, "_h", None):
            lib().airebo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st:
            raise AireboError(st, lib().airebo_last_error(self._h).decode())

    def _dev(self, t, dtype):
        t = t.to(device=self.device, dtype=dtype)
        return t.contiguous()

    def neighbor(self, pos, types, box):
        torch = self._torch
        pos = self._dev(pos, torch.float64)
        types = self._dev(types, torch.int8)
        assert pos.dim() == 2 and pos.shape[0] == 3 and pos.shape[1] == types.shape[0]
        b = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(3))
        self._check(lib().airebo_neighbor(self._h, _ptr(pos), _ptr(types), pos.shape[1], _np(b)))
        self.n = pos.shape[1]
        self._types = types
        self.box = b

    def neighbor_batch(self, pos, types, offsets, boxes):
        """Lists for independent systems: system s owns atoms offsets[s]:offsets[s+1]."""
        torch = self._torch
        pos = self._dev(pos, torch.float64)
        types = self._dev(types, torch.int8)
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        bx = np.ascontiguousarray(np.asarray(boxes, dtype=np.float64).reshape(-1, 3))
        self._check(lib().airebo_neighbor_batch(self._h, _ptr(pos), _ptr(types), pos.shape[1], len(off) - 1,
                                                _np(off), _np(bx)))
        self.n = pos.shape[1]
        self._types = types
        self.nsys = len(off) - 1

    def compute_batch(self, pos, force=None, energy=None):
        """Forces and the energy of each system."""
        torch = self._torch
        pos = self._dev(pos, torch.float64)
        if force is None:
            force = torch.empty_like(pos)
        if energy is None:
            energy = torch.empty(getattr(self, "nsys", 1), dtype=torch.float64, device=self.device)
        self._check(lib().airebo_compute_batch(self._h, _ptr(pos), _ptr(force), _ptr(energy)))
        return force, energy

    def compute_async(self, pos, force, energy4=None, energy_sys=None):
        self._check(lib().airebo_compute_async(self._h, _ptr(pos), _ptr(force), _ptr(energy4), _ptr(energy_sys)))

    def check(self):
        self._check(lib().airebo_check(self._h))

    def graph_capture(self, pos, force, energy4=None, energy_sys=None):
        """Capture one evaluation with these buffers into a CUDA graph."""
        self._check(lib().airebo_graph_capture(self._h, _ptr(pos), _ptr(force), _ptr(energy4), _ptr(energy_sys)))

    def autotune(self, pos, force=None):
        """Time the launch shapes on this system; returns (LJ atoms per warp claim, REBO/torsion waves,
        b* waves)."""
        torch = self._torch
        pos = self._dev(pos, torch.float64)
        if force is None:
            force = torch.empty_like(pos)
        out = np.zeros(3, dtype=np.int32)
        self._check(lib().airebo_autotune(self._h, _ptr(pos), _ptr(force), _np(out)))
        return int(out[0]), int(out[1]), int(out[2])

    def set_launch_shape(self, lj_chunk, bond_waves, bstar_waves):
        self._check(lib().airebo_set_launch_shape(self._h, int(lj_chunk), int(bond_waves), int(bstar_waves)))

    def graph_launch(self):
        self._check(lib().airebo_graph_launch(self._h))

    def compute(self, pos, force=None, virial=False, per_atom=False):
        """Forces (3, N), energies (total, REBO, LJ, torsion) and the virial (or None); with
        per_atom=True also the per-atom energies (N,) as a fourth value."""
        torch = self._torch
        pos = self._dev(pos, torch.float64)
        if force is None:
            force = torch.empty_like(pos)
        e4 = torch.empty(4, dtype=torch.float64, device=self.device)
        w6 = torch.empty(6, dtype=torch.float64, device=self.device) if virial else None
        ea = torch.empty(pos.shape[1], dtype=torch.float64, device=self.device) if per_atom else None
        self._check(lib().airebo_compute(self._h, _ptr(pos), _ptr(force), _ptr(e4), _ptr(w6), _ptr(ea)))
        if per_atom:
            return force, e4, w6, ea
        return force, e4, w6

    def param_grad(self, pos, force=None):
        """Forces, energies and dE/d(eps[3], sigma[3]) of the inter-molecular term."""
        torch = self._torch
        pos = self._dev(pos, torch.float64)
        if force is None:
            force = torch.empty_like(pos)
        e4 = torch.empty(4, dtype=torch.float64, device=self.device)
        g = np.zeros(6)
        self._check(lib().airebo_param_grad(self._h, _ptr(pos), _ptr(force), _ptr(e4), _np(g)))
        return force, e4, g

    def force_param_grad(self, pos, v, force=None):
        """Forces, energies and v . dF/d(eps[3], sigma[3]) for a direction v (3, N) on the device."""
        torch = self._torch
        pos = self._dev(pos, torch.float64)
        v = self._dev(v, torch.float64)
        if force is None:
            force = torch.empty_like(pos)
        e4 = torch.empty(4, dtype=torch.float64, device=self.device)
        g = np.zeros(6)
        self._check(lib().airebo_force_param_grad(self._h, _ptr(pos), _ptr(v), _ptr(force), _ptr(e4), _np(g)))
        return force, e4, g

    def knot_grad(self, pos, force=None):
        """Forces, energies and dE/d(spline knot data), KNOT_COUNT values in the parameter file's order."""
        torch = self._torch
        pos = self._dev(pos, torch.float64)
        if force is None:
            force = torch.empty_like(pos)
        e4 = torch.empty(4, dtype=torch.float64, device=self.device)
        g = np.zeros(KNOT_COUNT)
        self._check(lib().airebo_knot_grad(self._h, _ptr(pos), _ptr(force), _ptr(e4), _np(g), KNOT_COUNT))
        return force, e4, g

    def set_lj_params(self, eps=None, sigma=None):
        """Replace eps[3] and/or sigma[3]; a new sigma needs a new neighbor() call."""
        e = None if eps is None else np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(3))
        sg = None if sigma is None else np.ascontiguousarray(np.asarray(sigma, dtype=np.float64).reshape(3))
        self._check(lib().airebo_set_lj_params(self._h, _np(e), _np(sg)))

    def bstar_bound_check(self, pos):
        """The b* screen's bound on every queued pair: (bounded pairs, unbounded pairs, largest
        |b*_32 - b*_64| / bound, largest bound, pairs over their bound, largest difference)."""
        torch = self._torch
        pos = self._dev(pos, torch.float64)
        force = torch.empty_like(pos)
        out = np.zeros(6)
        self._check(lib().airebo_bstar_bound_check(self._h, _ptr(pos), _ptr(force), _np(out)))
        return dict(zip(("bounded", "unbounded", "max_ratio", "max_bound", "violations", "max_diff"), out.tolist()))

    def set_knots(self, knots):
        """Replace all KNOT_COUNT spline knot data (the order of knot_grad())."""
        k = np.ascontiguousarray(np.asarray(knots, dtype=np.float64).reshape(-1))
        self._check(lib().airebo_set_knots(self._h, _np(k), k.size))

    def needs_rebuild(self, pos) -> bool:
        flag = C.c_int(0)
        self._check(lib().airebo_needs_rebuild(self._h, _ptr(pos), C.byref(flag)))
        return bool(flag.value)

    def nve(self, pos, vel, force, dt: float, nsteps: int):
        """nsteps velocity-Verlet steps in place; returns (PE, KE, total, list builds)."""
        e4 = self._torch.empty(4, dtype=self._torch.float64, device=self.device)
        self._check(lib().airebo_nve(self._h, _ptr(pos), _ptr(vel), _ptr(force), dt, nsteps, _ptr(e4)))
        return e4

    def nve_async(self, pos, vel, force, dt: float, nsteps: int, energy4=None):
        """Enqueue nsteps NVE steps with the rebuild decided on the device (no host
        synchronisation); call check() afterwards.  Returns the energy buffer."""
        e4 = energy4 if energy4 is not None else self._torch.empty(4, dtype=self._torch.float64, device=self.device)
        self._check(lib().airebo_nve_async(self._h, _ptr(pos), _ptr(vel), _ptr(force), dt, nsteps, _ptr(e4)))
        return e4

    def graph_capture_nve(self, pos, vel, force, dt: float, nsteps: int, energy4=None):
        """Capture nsteps asynchronous NVE steps as this handle's graph; graph_launch() replays
        them.  Returns the energy buffer the graph writes (PE, KE, total, list builds)."""
        e4 = energy4 if energy4 is not None else self._torch.empty(4, dtype=self._torch.float64, device=self.device)
        self._check(lib().airebo_graph_capture_nve(self._h, _ptr(pos), _ptr(vel), _ptr(force), dt, nsteps, _ptr(e4)))
        return e4

    def compute_host(self, pos, types, box, virial=False, per_atom=False):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        types = np.ascontiguousarray(types, dtype=np.int8)
        b = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(3))
        n = types.shape[0]
        f = np.zeros((3, n))
        e4 = np.zeros(4)
        w6 = np.zeros(6) if virial else None
        ea = np.zeros(n) if per_atom else None
        self._check(lib().airebo_compute_host(self._h, _np(pos), _np(types), n, _np(b), _np(f), _np(e4), _np(w6),
                                              _np(ea)))
        self.n = n
        if per_atom:
            return f, e4, w6, ea
        return f, e4, w6

    def nve_host(self, pos, vel, force, dt: float, nsteps: int):
        """In-place NVE on host arrays (3, N) float64 (pinned or pageable)."""
        e4 = np.zeros(4)
        self._check(lib().airebo_nve_host(self._h, C.c_void_p(_addr(pos)), C.c_void_p(_addr(vel)),
                                          C.c_void_p(_addr(force)), dt, nsteps, _np(e4)))
        return e4

    def counters(self) -> dict:
        out = np.zeros(8, dtype=np.int64)
        self._check(lib().airebo_counters(self._h, _np(out)))
        names = ("bonds", "bstar", "bstar_dsb", "lj_in_cutoff", "map_cap", "list_builds", "lj_cap", "bstar_full")
        return dict(zip(names, out.tolist()))

    def export_lists(self, which: int, cap: int | None = None):
        """(counts, j, image) of list `which` (0 LJ half, 1 REBO intermediate, 2 exact REBO)."""
        n = self.n
        if cap is None:
            cap = {0: 2048, 1: 128, 2: 8}[which]
        cnt = np.zeros(n, dtype=np.int32)
        j = np.zeros((n, cap), dtype=np.int32)
        img = np.zeros((n, cap, 3), dtype=np.int8)
        self._check(lib().airebo_export_lists(self._h, which, _np(cnt), _np(j), _np(img), cap))
        return cnt, j, img

    def set_timing(self, on: bool = True):
        self._check(lib().airebo_set_timing(self._h, int(on)))

    def kernel_times(self) -> dict:
        ms = np.zeros(len(KERNELS))
        nl = np.zeros(len(KERNELS), dtype=np.int64)
        self._check(lib().airebo_kernel_times(self._h, _np(ms), _np(nl)))
        return {k: (float(ms[i]), int(nl[i])) for i, k in enumerate(KERNELS)}


class AireboEnergy:
    """Differentiable AIREBO energy:
    ``E = AireboEnergy.apply(pos, eps, sigma, evaluator, knots=None)``.

    The backward pass is the library's own force computation (F = -dE/dx);
    when eps or sigma (the three per-species-pair values of the
    inter-molecular term) require gradients, its hand-written dE/d(eps, sigma)
    (airebo_param_grad); when knots (a tensor of KNOT_COUNT spline knot data,
    the order of knot_grad()) is given and requires a gradient, its
    hand-written dE/d(knots) (airebo_knot_grad).  eps, sigma and knots are
    pushed to the evaluator before the evaluation; the neighbour lists are
    rebuilt each time."""

    _fn = None

    @classmethod
    def apply(cls, pos, eps, sigma, evaluator, knots=None):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, pos, eps, sigma, knots, ev):
                    ev.set_lj_params(eps.detach().cpu().numpy(), sigma.detach().cpu().numpy())
                    if knots is not None:
                        ev.set_knots(knots.detach().cpu().numpy())
                    ev.neighbor(pos.detach(), ev._types, ev.box)
                    need_p = ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
                    need_k = knots is not None and ctx.needs_input_grad[3]
                    if need_p:
                        f, e4, g = ev.param_grad(pos.detach())
                        gt = torch.tensor(g, dtype=torch.float64, device=pos.device)
                    else:
                        f, e4, _ = ev.compute(pos.detach())
                        gt = torch.zeros(6, dtype=torch.float64, device=pos.device)
                    gk = None
                    if need_k:
                        _, _, g = ev.knot_grad(pos.detach())
                        gk = torch.tensor(g, dtype=torch.float64, device=knots.device)
                    ctx.has_knots = knots is not None
                    ctx.save_for_backward(f, gt, gk)
                    return e4[0].clone()

                @staticmethod
                def backward(ctx, gE):
                    f, gt, gk = ctx.saved_tensors
                    gknots = gk * gE if (ctx.has_knots and gk is not None) else None
                    return -f * gE, gt[:3] * gE, gt[3:] * gE, gknots, None

            cls._fn = _F
        return cls._fn.apply(pos, eps, sigma, knots, evaluator)


class AireboForces:
    """Forces as a differentiable function of the inter-molecular parameters:
    ``F = AireboForces.apply(pos, eps, sigma, evaluator)`` (3, N), for
    force-matching losses such as sum |F - F_ref|^2.  The backward pass is the
    library's hand-written v . dF/d(eps, sigma) (airebo_force_param_grad) with
    v the incoming gradient of F; the gradient with respect to the positions
    (a Hessian-vector product) is not provided and raises when asked for."""

    _fn = None

    @classmethod
    def apply(cls, pos, eps, sigma, evaluator):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, pos, eps, sigma, ev):
                    ev.set_lj_params(eps.detach().cpu().numpy(), sigma.detach().cpu().numpy())
                    ev.neighbor(pos.detach(), ev._types, ev.box)
                    f, _, _ = ev.compute(pos.detach())
                    ctx.ev = ev
                    ctx.save_for_backward(pos.detach())
                    return f.clone()

                @staticmethod
                def backward(ctx, gF):
                    if ctx.needs_input_grad[0]:
                        raise NotImplementedError("AireboForces: no gradient with respect to the positions")
                    (pos,) = ctx.saved_tensors
                    _, _, g = ctx.ev.force_param_grad(pos, gF.contiguous())
                    gt = torch.tensor(g, dtype=torch.float64, device=pos.device)
                    return None, gt[:3], gt[3:], None

            cls._fn = _F
        return cls._fn.apply(pos, eps, sigma, evaluator)


def knot_vector(params: dict):
    """The KNOT_COUNT spline knot data of a parameter set, in the order of
    knot_grad() and set_knots()."""
    return np.concatenate([np.asarray(params[name], dtype=np.float64).ravel() for name, _ in KNOT_BLOCKS])


def _addr(a):
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data
