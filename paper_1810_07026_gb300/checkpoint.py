"""Checkpoints of an MD state: positions, velocities, species, box and step.

A checkpoint is one ``.npz`` file (NumPy's zip of arrays), written and read
on the host; a run resumed from it continues exactly where the saved one
stopped (the integrator keeps no other state: the lists are rebuilt at the
first step).  The paper replays runs from trace dumps (Sec. 3.3); these files
serve the same purpose for the GPU path.
"""
from __future__ import annotations

import numpy as np

FORMAT = 1


def save(path: str, pos, vel, types, box, step: int, meta: dict | None = None) -> None:
    """Write pos (3, N), vel (3, N) float64, types (N,) int8, box (3,) and the step number."""
    def host(a, dtype):
        if hasattr(a, "detach"):
            a = a.detach().cpu().numpy()
        return np.ascontiguousarray(np.asarray(a, dtype=dtype))
    pos = host(pos, np.float64)
    vel = host(vel, np.float64)
    types = host(types, np.int8)
    box = host(box, np.float64).reshape(3)
    if pos.shape != vel.shape or pos.ndim != 2 or pos.shape[0] != 3 or pos.shape[1] != types.shape[0]:
        raise ValueError("pos and vel must be (3, N) and types (N,)")
    extra = {f"meta_{k}": np.asarray(v) for k, v in (meta or {}).items()}
    np.savez(path, format=np.int64(FORMAT), pos=pos, vel=vel, types=types, box=box, step=np.int64(step), **extra)


def load(path: str) -> dict:
    """The arrays of a checkpoint (host NumPy): pos, vel, types, box, step, meta."""
    with np.load(path) as z:
        if int(z["format"]) != FORMAT:
            raise ValueError(f"unknown checkpoint format {int(z['format'])}")
        meta = {k[5:]: z[k] for k in z.files if k.startswith("meta_")}
        return dict(pos=z["pos"].copy(), vel=z["vel"].copy(), types=z["types"].copy(), box=z["box"].copy(),
                    step=int(z["step"]), meta=meta)
