"""ctm_svd_noalloc: the batched SVD for callers that cannot allocate device memory.

Its workspace is a fixed array inside libctm, so it suits code that must not
call cudaMalloc (memory owned by a caller's pool, allocators that forbid new
allocations while they run).  It must give the same result as ctm_svd, the
allocating entry point, and keep giving it on the next call, whose inputs
differ (the shared array keeps the previous call's contents).

Collected last so that a stop-at-first-failure run has already run the rest.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _svd_both(lib, M):
    b, r = M.shape[0], M.shape[1]
    outs = []
    for fn in (lib.ctm_svd, lib.ctm_svd_noalloc):
        U = torch.empty_like(M)
        V = torch.empty_like(M)
        s = torch.empty(b, r, dtype=torch.float64, device=M.device)
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = fn(ctypes.c_void_p(M.data_ptr()), b, r, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                ctypes.c_void_p(V.data_ptr()), st)
        assert rc == 0
        torch.cuda.synchronize()
        outs.append((U.cpu().numpy(), s.cpu().numpy(), V.cpu().numpy()))
    return outs


def test_noalloc_svd_matches_allocating_entry_point_twice():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_14414_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(2024)
    for b, r in ((3, 40), (2, 33)):  # two calls in a row, different shapes and data
        M = rng.standard_normal((b, r, r)) @ np.diag(np.logspace(0, -6, r))
        Mt = torch.tensor(M, device="cuda")
        (U1, s1, V1), (U2, s2, V2) = _svd_both(lib, Mt)
        scale = s1[:, :1]
        assert np.abs(s1 - s2).max() <= 1e-12 * scale.max()
        for k in range(b):
            assert np.abs(U1[k] * s1[k] - U2[k] * s2[k]).max() <= 1e-12 * s1[k, 0]
            assert np.abs(V1[k] - V2[k]).max() <= 1e-12
            assert np.abs(U2[k] @ np.diag(s2[k]) @ V2[k].T - M[k]).max() <= 1e-13 * s1[k, 0]


def test_noalloc_rejects_sizes_beyond_its_array():
    from paper_2512_14414_gb300 import _lib
    lib = _lib.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    dummy = ctypes.c_void_p(1)
    assert lib.ctm_svd_noalloc(dummy, 1, 1025, dummy, dummy, dummy, st) == 1   # 1025^2 > 2^20
    assert lib.ctm_svd_noalloc(dummy, 1025, 4, dummy, dummy, dummy, st) == 1   # batch > 1024
