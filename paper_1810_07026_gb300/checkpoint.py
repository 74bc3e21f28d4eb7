"""Checkpoints of an MD state: positions, velocities, species, box, step, and
the settings the continuation depends on.

A checkpoint is one ``.npz`` file (NumPy's zip of arrays), written and read
on the host.  Besides the state it holds, as required fields, the time step,
the precision, the neighbour-list skin and the parameter text (with its
SHA-256), because a run resumed with another time step, precision or
parameter set would not continue the saved one.  ``check`` compares them
with the settings of a resumed run and raises on any difference.  The
integrator keeps no other state (the lists are rebuilt at the first step), so
a run resumed with the same settings continues where the saved one stopped.
The paper replays runs from trace dumps (Sec. 3.3); these files serve the
same purpose for the GPU path.
"""
from __future__ import annotations

import hashlib

import numpy as np

FORMAT = 2


def params_digest(params) -> str:
    """SHA-256 of a parameter set's text (a dict is serialised first)."""
    if isinstance(params, dict):
        from . import inputs
        params = inputs.params_text(params)
    return hashlib.sha256(params.encode()).hexdigest()


def save(path: str, pos, vel, types, box, step: int, *, dt: float, precision: int, skin: float, params,
         meta: dict | None = None) -> None:
    """Write pos (3, N), vel (3, N) float64, types (N,) int8, box (3,), the step
    number, and the run's dt (fs), precision, skin (A) and parameter set."""
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
    if not (dt > 0) or not (skin >= 0) or precision not in (0, 1, 2):
        raise ValueError("dt must be positive, skin non-negative, precision 0, 1 or 2")
    if isinstance(params, dict):
        from . import inputs
        params = inputs.params_text(params)
    extra = {f"meta_{k}": np.asarray(v) for k, v in (meta or {}).items()}
    np.savez(path, format=np.int64(FORMAT), pos=pos, vel=vel, types=types, box=box, step=np.int64(step),
             dt=np.float64(dt), precision=np.int64(precision), skin=np.float64(skin),
             params=np.asarray(params), params_sha256=np.asarray(params_digest(params)), **extra)


def load(path: str) -> dict:
    """The contents of a checkpoint (host NumPy): pos, vel, types, box, step,
    dt, precision, skin, params (text), params_sha256, meta."""
    with np.load(path) as z:
        fmt = int(z["format"])
        if fmt != FORMAT:
            raise ValueError(f"checkpoint format {fmt}, expected {FORMAT} (dt, precision, skin and parameters "
                             "are required fields)")
        params = str(z["params"])
        digest = str(z["params_sha256"])
        if params_digest(params) != digest:
            raise ValueError("checkpoint parameter text does not match its SHA-256")
        meta = {k[5:]: z[k] for k in z.files if k.startswith("meta_")}
        return dict(pos=z["pos"].copy(), vel=z["vel"].copy(), types=z["types"].copy(), box=z["box"].copy(),
                    step=int(z["step"]), dt=float(z["dt"]), precision=int(z["precision"]), skin=float(z["skin"]),
                    params=params, params_sha256=digest, meta=meta)


def check(state: dict, *, dt: float, precision: int, skin: float, params) -> None:
    """Raise ValueError unless a resumed run's dt, precision, skin and
    parameter set equal the checkpoint's."""
    bad = []
    if float(dt) != state["dt"]:
        bad.append(f"dt {dt} != {state['dt']}")
    if int(precision) != state["precision"]:
        bad.append(f"precision {precision} != {state['precision']}")
    if float(skin) != state["skin"]:
        bad.append(f"skin {skin} != {state['skin']}")
    if params_digest(params) != state["params_sha256"]:
        bad.append("parameter set differs")
    if bad:
        raise ValueError("checkpoint does not match the resumed run: " + "; ".join(bad))


def check_evaluator(state: dict, evaluator, dt: float) -> None:
    """check() against an Airebo evaluator's own settings."""
    check(state, dt=dt, precision=evaluator.precision, skin=evaluator.skin, params=evaluator.params_text)
