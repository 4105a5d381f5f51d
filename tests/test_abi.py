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


def _desc(lib_mod, Lx=1, Ly=1, d=2, D=2, chi=4, precision=0, terms=None, n_terms=None):
    import numpy as np
    hm = np.eye(d * d)
    if terms is None:
        terms = [(0, 0, 0)]
    arr = (lib_mod.CtmTerm * max(1, len(terms)))()
    for k, (x, y, kind) in enumerate(terms):
        arr[k].x, arr[k].y, arr[k].kind, arr[k].coupling = x, y, kind, 1.0
        arr[k].h = hm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    desc = lib_mod.CtmDesc(Lx, Ly, d, D, chi, precision, len(terms) if n_terms is None else n_terms, arr, 0.0, -1.0, 0)
    return desc, arr, hm


def test_create_rejects_each_bad_description_without_gpu():
    from paper_2512_14414_gb300 import _lib
    lib = _lib.load()
    h = ctypes.c_void_p()
    bad = [dict(chi=0), dict(D=0), dict(Lx=0), dict(precision=5), dict(precision=-1),
           dict(terms=[(1, 0, 0)]), dict(terms=[(0, 0, 4)]), dict(n_terms=65),
           dict(D=9, chi=128)]  # chi * D * d = 2304 > 2048
    for kw in bad:
        desc, arr, hm = _desc(_lib, **kw)
        assert lib.ctm_create(ctypes.byref(desc), ctypes.byref(h)) == 1, kw
    for prec in range(5):  # every precision mode, and the largest bond that fits (81 * 9 * 2 = 1458)
        desc, arr, hm = _desc(_lib, D=9, chi=81, precision=prec)
        assert lib.ctm_create(ctypes.byref(desc), ctypes.byref(h)) == 0
        assert lib.ctm_destroy(h) == 0


def test_stateless_entry_points_check_their_arguments_without_gpu():
    from paper_2512_14414_gb300 import _lib
    lib = _lib.load()
    vp = ctypes.c_void_p
    one = vp(1)
    # batched SVD: null matrices, empty batch, oversize
    assert lib.ctm_svd(None, 1, 4, one, one, one, None) == 1
    assert lib.ctm_svd(one, 0, 4, one, one, one, None) == 1
    assert lib.ctm_svd(one, 1, 5000, one, one, one, None) == 1
    # allocation-free SVD: beyond its fixed array (batch <= 1024, batch * r * r <= 2^20)
    assert lib.ctm_svd_noalloc(one, 1025, 4, one, one, one, None) == 1
    assert lib.ctm_svd_noalloc(one, 2, 1024, one, one, one, None) == 1
    # MLP forward: null input, no layers, too many layers, an empty width
    dims = (ctypes.c_int * 3)(4, 8, 2)
    W = (vp * 2)(1, 1)
    assert lib.ctm_mlp_forward(None, 1, 2, dims, W, None, one, one, None) == 1
    assert lib.ctm_mlp_forward(one, 1, 0, dims, W, None, one, one, None) == 1
    assert lib.ctm_mlp_forward(one, 1, 17, dims, W, None, one, one, None) == 1
    dims0 = (ctypes.c_int * 3)(4, 0, 2)
    assert lib.ctm_mlp_forward(one, 1, 2, dims0, W, None, one, one, None) == 1
    assert lib.ctm_mlp_forward(one, 0, 2, dims, W, None, one, one, None) == 1


def test_mlp_work_size_and_training_argument_checks_without_gpu():
    # host-only entry points of the warm-start training: the work size follows its layout (the
    # hidden layers' pre-activations and activations, the output, two gradient buffers and 1024
    # partial sums), and bad arguments are refused before any device work
    from paper_2512_14414_gb300 import _lib
    lib = _lib.load()
    dims = (ctypes.c_int * 5)(32, 1024, 1024, 1024, 200)
    batch = 8
    expect = 2 * batch * 1024 * 3 + batch * 200 + 2 * batch * 1024 + 1024
    assert lib.ctm_mlp_work_floats(batch, 4, dims) == expect
    assert lib.ctm_mlp_work_floats(0, 4, dims) == -1
    bad = (ctypes.c_int * 3)(4, 0, 2)
    assert lib.ctm_mlp_work_floats(1, 2, bad) == -1
    vp = ctypes.c_void_p
    assert lib.ctm_mlp_backward(None, None, batch, 4, dims, None, None, None, None, None, None, None) == 1
    assert lib.ctm_adam_step(None, None, None, None, 10, 1e-3, 0.9, 0.999, 1e-8, 1, None) == 1
    assert lib.ctm_adam_step(vp(8), vp(8), vp(8), vp(8), 10, 1e-3, 0.9, 0.999, 1e-8, 0, None) == 1  # t < 1
    assert lib.ctm_adam_step(vp(8), vp(8), vp(8), vp(8), 10, 1e-3, 1.0, 0.999, 1e-8, 1, None) == 1  # beta1 = 1
