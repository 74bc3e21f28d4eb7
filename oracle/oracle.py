"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

Builds ``oracle/liboracle.so`` from ``airebo_oracle.cpp`` with g++ (OpenMP)
and wraps its entry points with numpy arrays.  Only the tests, the smoke check
and the bench's CPU baseline use it; the library under test never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "airebo_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

FLAG_REBO, FLAG_LJ, FLAG_TORSION = 1, 2, 4
FLAG_ALL = 7
COUNTERS = ("bonds", "bo_nbr_terms", "dihedral_pairs", "torsion_quads", "lj_candidates",
            "lj_in_cutoff", "lj_c_zero", "bstar", "bstar_dsb_nonzero", "paths")

_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", "-o", LIB + ".tmp", SRC]
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.c_void_p
        L.oracle_create.restype = P
        L.oracle_create.argtypes = [C.c_char_p]
        L.oracle_destroy.argtypes = [P]
        L.oracle_threads.restype = C.c_int
        L.oracle_set_threads.argtypes = [C.c_int]
        L.oracle_compute_masked.restype = C.c_int
        L.oracle_compute_masked.argtypes = [P, C.c_int64, P, P, P, C.c_int, P, P, P, P, P, P, P, P]
        L.oracle_compute.restype = C.c_int
        L.oracle_compute.argtypes = [P, C.c_int64, P, P, P, C.c_int, P, P, P, P, P]
        for f in (L.oracle_rebo_neighbors, L.oracle_lj_pairs):
            f.restype = C.c_int64
            f.argtypes = [P, C.c_int64, P, P, P, C.c_int64, P, P, P]
        L.oracle_cij.restype = C.c_double
        L.oracle_cij.argtypes = [P, C.c_int64, C.c_int64, P, P]
        L.oracle_spline.restype = C.c_double
        L.oracle_spline.argtypes = [P, C.c_int, C.c_double, C.c_double, C.c_double, P]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class Oracle:
    """The FP64 oracle for one parameter set."""

    def __init__(self, param_text: str):
        self._h = lib().oracle_create(param_text.encode())
        if not self._h:
            raise ValueError("oracle: could not parse parameter text")

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.oracle_destroy(self._h)
            self._h = None

    @staticmethod
    def _sys(pos, types, box):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        types = np.ascontiguousarray(types, dtype=np.int8)
        box = np.ascontiguousarray(box, dtype=np.float64)
        assert pos.shape[0] == 3 and pos.shape[1] == types.shape[0]
        return pos, types, box

    def compute(self, pos, types, box, flags=FLAG_ALL, forces=True, per_atom=False):
        """Energy (total, REBO, LJ, torsion), forces (3, N), virial (6,), counters; with
        per_atom=True also the per-atom energies (N,), each term split evenly between its i and j."""
        pos, types, box = self._sys(pos, types, box)
        n = types.shape[0]
        f = np.zeros((3, n)) if forces else None
        e = np.zeros(4)
        w = np.zeros(6)
        c = np.zeros(16, dtype=np.int64)
        ea = np.zeros(n) if per_atom else None
        lib().oracle_compute(self._h, n, _ptr(pos), _ptr(types), _ptr(box), flags, _ptr(f), _ptr(e), _ptr(w), _ptr(c),
                             _ptr(ea))
        if per_atom:
            return e, f, w, dict(zip(COUNTERS, c.tolist())), ea
        return e, f, w, dict(zip(COUNTERS, c.tolist()))

    def energy(self, pos, types, box, flags=FLAG_ALL):
        return self.compute(pos, types, box, flags, forces=False)[0][0]

    def forces_subset(self, pos, types, box, atoms, flags=FLAG_ALL, radius=None, counters=False):
        """Forces on the listed atoms only, from the terms anchored near them.

        Every term that can touch an atom is anchored at an atom within
        `radius` of it (default: the LJ cut-off plus four REBO bond lengths),
        so the forces are complete for the selected atoms.  Neighbour sets
        are built only where those terms look."""
        pos, types, box = self._sys(pos, types, box)
        n = types.shape[0]
        atoms = np.asarray(atoms, dtype=np.int64)
        if radius is None:
            radius = 3.0 * 3.40 + 4 * 2.0 + 0.5
        sel = np.zeros(n, dtype=np.int8)
        sel[atoms] = 1
        anchor = np.zeros(n, dtype=np.int8)
        need = np.zeros(n, dtype=np.int8)
        for a in atoms:
            d = pos - pos[:, a:a + 1]
            d -= box[:, None] * np.round(d / box[:, None])
            r2 = np.einsum("ij,ij->j", d, d)
            anchor[r2 < radius * radius] = 1
            need[r2 < (radius + 8.5) ** 2] = 1
        f = np.zeros((3, n))
        c = np.zeros(16, dtype=np.int64)
        lib().oracle_compute_masked(self._h, n, _ptr(pos), _ptr(types), _ptr(box), flags, _ptr(anchor), _ptr(sel),
                                    _ptr(need), _ptr(f), None, None, _ptr(c), None)
        if counters:
            return f[:, atoms], dict(zip(COUNTERS, c.tolist()))
        return f[:, atoms]

    def evaluate_sphere(self, pos, types, box, center, radius, flags=FLAG_ALL):
        """Energy, forces and counters of all terms anchored at the atoms within
        `radius` of atom `center` (minimum image): a bounded sample of a large
        system.  Returns (energy4, forces on all atoms, counters, anchor count)."""
        pos, types, box = self._sys(pos, types, box)
        n = types.shape[0]
        d = pos - pos[:, center:center + 1]
        d -= box[:, None] * np.round(d / box[:, None])
        r2 = np.einsum("ij,ij->j", d, d)
        anchor = (r2 < radius * radius).astype(np.int8)
        need = (r2 < (radius + 20.0) ** 2).astype(np.int8)
        f = np.zeros((3, n))
        e = np.zeros(4)
        c = np.zeros(16, dtype=np.int64)
        lib().oracle_compute_masked(self._h, n, _ptr(pos), _ptr(types), _ptr(box), flags, _ptr(anchor), None,
                                    _ptr(need), _ptr(f), _ptr(e), None, _ptr(c), None)
        return e, f, dict(zip(COUNTERS, c.tolist())), int(anchor.sum())

    def _pairs(self, fn, pos, types, box, cap=None):
        pos, types, box = self._sys(pos, types, box)
        n = types.shape[0]
        cap = cap or 400 * n + 16
        j = np.zeros(cap, dtype=np.int32)
        img = np.zeros((cap, 3), dtype=np.int8)
        off = np.zeros(n + 1, dtype=np.int64)
        c = fn(self._h, n, _ptr(pos), _ptr(types), _ptr(box), cap, _ptr(j), _ptr(img), _ptr(off))
        if c < 0:
            raise RuntimeError("pair capacity too small")
        return off, j[:c], img[:c]

    def rebo_neighbors(self, pos, types, box):
        return self._pairs(lib().oracle_rebo_neighbors, pos, types, box)

    def lj_pairs(self, pos, types, box):
        return self._pairs(lib().oracle_lj_pairs, pos, types, box)

    def cij(self, i, j, img):
        """C_ij of a pair; call rebo_neighbors or compute on the system first."""
        im = np.asarray(img, dtype=np.int32)
        path = np.zeros(3, dtype=np.int32)
        c = lib().oracle_cij(self._h, int(i), int(j), _ptr(im), _ptr(path))
        return c, tuple(path.tolist())

    def spline(self, which, x, y=0.0, z=0.0):
        g = np.zeros(3)
        v = lib().oracle_spline(self._h, which, x, y, z, _ptr(g))
        return v, g


def threads() -> int:
    return int(lib().oracle_threads())


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))
