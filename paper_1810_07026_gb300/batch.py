"""Batched independent systems: relaxation of a random ensemble on the GPU path.

The ensemble's random insertion leaves atoms 1 A apart; 200 steps of FP64
steepest descent (each atom's step capped at 0.1 A) on the library's forces
take it to a less strained, still amorphous state before it is used.  Every
force comes from the CUDA library; only the position update is done here.
"""
from __future__ import annotations

from . import airebo


def relax(params, pos, types, offsets, boxes, steps: int = 200, alpha: float = 0.01, cap: float = 0.1):
    """Steepest descent x += alpha F (A^2/eV), each atom's step at most `cap` A.
    pos: torch (3, N) float64 on the device, updated in place.  Returns the
    per-system energies after the last step."""
    import torch
    ev = airebo.Airebo(params, precision=airebo.FP64)
    ev.neighbor_batch(pos, types, offsets, boxes)
    e = None
    for _ in range(steps):
        f, e = ev.compute_batch(pos)
        step = alpha * f
        scale = torch.clamp(cap / step.norm(dim=0).clamp_min(1e-30), max=1.0)
        pos += step * scale
        if ev.needs_rebuild(pos):
            ev.neighbor_batch(pos, types, offsets, boxes)
    f, e = ev.compute_batch(pos)
    ev.close()
    return e
