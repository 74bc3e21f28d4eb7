"""The rebuild check that allocates no device memory, through the C ABI.

It serves callers that cannot call cudaMalloc (code inside a framework that
owns all device memory, or code that must not allocate after set-up).  Its
answer must equal airebo_needs_rebuild's on the same positions, and its
maximum displacement must equal the plain definition max |x - x_ref|, on two
calls in a row (the scratch array keeps the first call's contents).  This
file is collected last so that a failure here comes after every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1810_07026_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def call_noalloc(lib, pos, ref, n, skin, stream):
    flag = C.c_int(-1)
    maxd = C.c_double(-1.0)
    st = lib.airebo_needs_rebuild_noalloc(C.c_void_p(pos.data_ptr()), C.c_void_p(ref.data_ptr()), C.c_int64(n),
                                          C.c_double(skin), C.c_void_p(stream), C.byref(flag), C.byref(maxd))
    return st, flag.value, maxd.value


def test_noalloc_rebuild_check_matches_existing_entry_point():
    from paper_1810_07026_gb300 import build, airebo
    build.build()
    lib = airebo.lib()
    lib.airebo_needs_rebuild_noalloc.restype = C.c_int
    lib.airebo_needs_rebuild_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_void_p,
                                                 C.c_void_p, C.c_void_p]
    skin = 1.0
    pos, types, box = inputs.polyethylene(6, 8, 16, noise=0.05)      # 9,216 atoms
    n = len(types)
    ev = airebo.Airebo(inputs.make_params(0), skin=skin)
    ref = torch.tensor(pos, device="cuda")
    ev.neighbor(ref, torch.tensor(types, device="cuda"), box)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(9)
    # two calls in a row: one below skin/2, one above
    for amp in (0.2, 1.6):
        d = rng.normal(0.0, 1.0, (3, n))
        d *= amp * 0.5 * skin / np.linalg.norm(d, axis=0).max()
        p = ref + torch.tensor(d, device="cuda")
        torch.cuda.synchronize()
        st, flag, maxd = call_noalloc(lib, p, ref, n, skin, stream)
        assert st == 0
        assert flag == int(ev.needs_rebuild(p))
        want = np.linalg.norm(d, axis=0).max()
        assert maxd == pytest.approx(want, rel=1e-12)
        assert flag == int(amp > 1.0)


def _lib():
    from paper_1810_07026_gb300 import build, airebo
    build.build()
    lib = airebo.lib()
    lib.airebo_needs_rebuild_noalloc.restype = C.c_int
    lib.airebo_needs_rebuild_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_void_p,
                                                 C.c_void_p, C.c_void_p]
    return lib


def test_noalloc_ragged_tail_matches_existing_entry_point():
    """n = 9,000 (not a multiple of the 256-atom blocks: the last block is
    partly empty) on contiguous (3, n) copies; the largest displacement is put
    in the ragged tail so that the tail must be read."""
    from paper_1810_07026_gb300 import airebo
    lib = _lib()
    skin = 1.0
    pos, types, box = inputs.polyethylene(6, 8, 16, noise=0.05)
    n = 9000
    pos, types = np.ascontiguousarray(pos[:, :n]), np.ascontiguousarray(types[:n])
    ev = airebo.Airebo(inputs.make_params(0), skin=skin)
    ref = torch.tensor(pos, device="cuda")
    ev.neighbor(ref, torch.tensor(types, device="cuda"), box)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(3)
    for amp, at in ((0.3, n - 1), (1.4, n - 5)):
        d = rng.normal(0.0, 1.0, (3, n))
        d *= 0.1 * 0.5 * skin / np.linalg.norm(d, axis=0).max()
        d[:, at] = [amp * 0.5 * skin, 0.0, 0.0]
        p = ref + torch.tensor(d, device="cuda")
        torch.cuda.synchronize()
        st, flag, maxd = call_noalloc(lib, p, ref, n, skin, stream)
        assert st == 0
        assert flag == int(ev.needs_rebuild(p)) == int(amp > 1.0)
        assert maxd == pytest.approx(np.linalg.norm(d, axis=0).max(), rel=1e-12)


def test_noalloc_largest_size():
    """n = 2,097,152 atoms, the most the scratch array allows (8,192 blocks,
    every slot of the block maxima in use), against the maximum on the host."""
    lib = _lib()
    n = 2_097_152
    g = torch.Generator(device="cuda").manual_seed(11)
    ref = torch.rand((3, n), dtype=torch.float64, device="cuda", generator=g) * 100.0
    stream = torch.cuda.current_stream().cuda_stream
    for scale in (0.2, 0.9):
        d = (torch.rand((3, n), dtype=torch.float64, device="cuda", generator=g) - 0.5) * scale
        p = ref + d
        torch.cuda.synchronize()
        st, flag, maxd = call_noalloc(lib, p, ref, n, 1.0, stream)
        assert st == 0
        dh = (p - ref).cpu().numpy()
        want = np.sqrt((dh * dh).sum(axis=0)).max()
        assert maxd == pytest.approx(want, rel=1e-12)
        assert flag == int(want > 0.5)
    del p, ref, d
    torch.cuda.empty_cache()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1810_07026_gb300 import build, airebo
    build.build()
    lib = airebo.lib()
    lib.airebo_needs_rebuild_noalloc.restype = C.c_int
    flag = C.c_int(-1)
    st = lib.airebo_needs_rebuild_noalloc(C.c_void_p(1), C.c_void_p(1), C.c_int64(2_097_153), C.c_double(1.0),
                                          None, C.byref(flag), None)
    assert st == airebo.ERR_ARG and flag.value == -1
