"""Checkpoint files round-trip the MD state exactly and refuse a resumed run
with other settings (host only)."""
import numpy as np
import pytest

from paper_1810_07026_gb300 import checkpoint, inputs


def _state(tmp_path):
    pos, types, box = inputs.polyethylene(2, 2, 3, noise=0.03)
    vel = inputs.velocities(types, 300.0, seed=3)
    text = inputs.params_text(inputs.make_params(0))
    f = tmp_path / "state.npz"
    checkpoint.save(str(f), pos, vel, types, box, 17, dt=0.5, precision=0, skin=1.0, params=text,
                    meta={"note": "x"})
    return f, pos, vel, types, box, text


def test_round_trip(tmp_path):
    f, pos, vel, types, box, text = _state(tmp_path)
    s = checkpoint.load(str(f))
    assert np.array_equal(s["pos"], pos) and np.array_equal(s["vel"], vel)
    assert np.array_equal(s["types"], types.astype(np.int8)) and np.array_equal(s["box"], np.asarray(box, float))
    assert s["step"] == 17 and s["dt"] == 0.5 and s["precision"] == 0 and s["skin"] == 1.0
    assert s["params"] == text and str(s["meta"]["note"]) == "x"
    checkpoint.check(s, dt=0.5, precision=0, skin=1.0, params=text)


@pytest.mark.parametrize("change", ["dt", "precision", "skin", "params"])
def test_mismatch_raises(tmp_path, change):
    f, _, _, _, _, text = _state(tmp_path)
    s = checkpoint.load(str(f))
    kw = dict(dt=0.5, precision=0, skin=1.0, params=text)
    kw[change] = {"dt": 0.25, "precision": 1, "skin": 2.0, "params": inputs.make_params(1)}[change]
    with pytest.raises(ValueError, match="does not match"):
        checkpoint.check(s, **kw)


def test_required_fields_and_format(tmp_path):
    pos, types, box = inputs.diamond()
    with pytest.raises(TypeError):
        checkpoint.save(str(tmp_path / "x.npz"), pos, pos, types, box, 0)
    with pytest.raises(ValueError):
        checkpoint.save(str(tmp_path / "x.npz"), pos, pos[:, :5], types, box, 0, dt=0.5, precision=0, skin=1.0,
                        params="p 1 1")
    old = tmp_path / "old.npz"
    np.savez(old, format=np.int64(1), pos=pos, vel=pos, types=types, box=box, step=np.int64(0))
    with pytest.raises(ValueError, match="format"):
        checkpoint.load(str(old))
