"""Checkpoint files round-trip the MD state exactly (host only)."""
import numpy as np
import pytest

from paper_1810_07026_gb300 import checkpoint, inputs


def test_round_trip(tmp_path):
    pos, types, box = inputs.polyethylene(2, 2, 3, noise=0.03)
    vel = inputs.velocities(types, 300.0, seed=3)
    f = tmp_path / "state.npz"
    checkpoint.save(str(f), pos, vel, types, box, 17, meta={"dt": 0.5})
    s = checkpoint.load(str(f))
    assert np.array_equal(s["pos"], pos) and np.array_equal(s["vel"], vel)
    assert np.array_equal(s["types"], types.astype(np.int8)) and np.array_equal(s["box"], np.asarray(box, float))
    assert s["step"] == 17 and float(s["meta"]["dt"]) == 0.5


def test_rejects_bad_shapes(tmp_path):
    pos, types, box = inputs.diamond()
    with pytest.raises(ValueError):
        checkpoint.save(str(tmp_path / "x.npz"), pos, pos[:, :5], types, box, 0)
