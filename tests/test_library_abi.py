"""The C-ABI library loads and exports every function include/airebo.h declares (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "airebo.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(airebo_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_1810_07026_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_default_options_without_gpu():
    from paper_1810_07026_gb300 import build, airebo
    build.build()
    opt = airebo.Options()
    airebo.lib().airebo_default_options(ctypes.byref(opt))
    assert opt.skin == 1.0 and opt.precision == 0 and opt.enable_lj == 1 and opt.max_lj_nbrs == 0
