"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ctm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|const char\*)\s+(ctm_\w+)\s*\(", src, re.M)))


def test_build_and_exports():
    import __graft_entry__ as g
    g.build()
    from paper_2512_14414_gb300 import _lib
    lib = ctypes.CDLL(_lib.LIB_PATH)
    syms = declared_symbols()
    assert len(syms) >= 10
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(_lib.EXPORTS) == syms


def test_error_strings_and_argument_checks_without_gpu():
    from paper_2512_14414_gb300 import _lib
    lib = _lib.load()
    assert lib.ctm_error_string(0) == b"ok"
    assert lib.ctm_error_string(5) == b"SVD did not converge"
    h = ctypes.c_void_p()
    assert lib.ctm_create(None, ctypes.byref(h)) == 1          # INVALID_ARG, host-side only
    desc = _lib.CtmDesc(1, 1, 2, 2, 4, 0, 0, None, 1e-6, 1e-30, 0)
    assert lib.ctm_create(ctypes.byref(desc), ctypes.byref(h)) == 1   # no terms
    import numpy as np
    hm = np.eye(4)
    t = (_lib.CtmTerm * 1)()
    t[0].x, t[0].y, t[0].kind, t[0].coupling = 0, 0, 0, 1.0
    t[0].h = hm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    desc = _lib.CtmDesc(1, 1, 2, 2, 4, 0, 1, t, 1e-6, 1e-30, 0)
    assert lib.ctm_create(ctypes.byref(desc), ctypes.byref(h)) == 0
    import workloads as W
    expect = sum(int(np.prod(shp)) for site in W.env_shapes(1, 1, 2, 2, 4) for shp in site)
    assert lib.ctm_env_numel(h) == expect
    assert lib.ctm_step(h, 1, None, None) == 8                 # STATE: not initialised
    assert lib.ctm_destroy(h) == 0
